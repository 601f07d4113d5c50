"""Learned proposal on the GPU against the float64 oracle (oracle/mdn.py).

Network: forward outputs and the loss within BF16 tolerances, gradients of every layer
against the oracle's backward pass, Adam against the oracle's update, training that
lowers the loss and is bitwise deterministic. Mixture arithmetic used by the sampler:
densities and inverse-CDF draws in FP64 (1e-12) and mixed precision.

Tolerances. BF16 keeps 8 significant bits (unit roundoff u = 2^-9 = 2e-3). The tensor-core
network rounds every weight matrix and hidden activation to BF16; the oracle's
``quantized`` network applies the same roundings and computes everything else in float64,
so the forward outputs agree to float32 accumulation error (held to 1e-4), and against the
unrounded float64 network to a few u over four layers (held to 1e-2). The backward pass
keeps the back-propagated signal as a BF16 pair hi + lo (~16 bits) and accumulates in
float32, so on its own it adds ~1e-4; what remains on a random batch comes from the forward
pass: float32 and float64 accumulation put a pre-activation within ~1e-4 of zero on
opposite sides of the ReLU kink now and then, and each such flip moves one whole term of a
batch sum whose terms largely cancel (~1e-2 at 1000 rows, growing with the batch). Hence
two gradient tests: every row of a random batch against 1e-2, and the rows whose
pre-activations all keep 1e-3 of their RMS away from zero (chosen from the oracle's forward
pass) against 1e-3. The loss, a batch mean, to 1e-3.
The gradient of the quantized network differs from the unrounded network's by up to ~7%
on the first layer: the two are gradients of different functions, and the trained
function is the quantized one.
"""
import numpy as np
import pytest

from oracle import mdn as MD

from _common import rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _bf16(a):
    return MD.to_bf16(a)


def _setup(torch, g, B, scale=1.0):
    theta = MD.init_params(g, scale=scale).astype(np.float32).astype(np.float64)
    x = _bf16(g.normal(0, 1, (B, MD.N_IN)))
    dev = torch.device("cuda")
    pt = torch.from_numpy(theta.astype(np.float32)).to(dev)
    xt = torch.from_numpy(x.astype(np.float32)).to(dev).to(torch.bfloat16)
    assert np.array_equal(xt.float().cpu().numpy().astype(np.float64), x)
    return theta, x, pt, xt


@pytest.mark.parametrize("B", [300, 4100])
def test_forward_matches_oracle(B):
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = np.random.default_rng(B)
    theta, x, pt, xt = _setup(torch, g, B)
    net = L.Mdn(B)
    L.mdn_set_params(net, pt)
    raw = torch.full((B, MD.N_OUT), float("nan"), dtype=torch.float32, device="cuda")
    L.mdn_forward(net, xt, raw)
    L.mdn_status(net)
    got = raw.cpu().numpy().astype(np.float64)
    want, _ = MD.forward(theta, x)
    assert np.all(np.isfinite(got))
    err = rel_l2(got, want)
    assert err < 1e-2, err
    wq, _ = MD.forward(theta, x, quantized=True)
    assert rel_l2(got, wq) < 1e-4, rel_l2(got, wq)
    # every row, not only the bulk (ragged last tiles)
    rows = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert rows.max() < 3e-2, rows.max()
    net.close()


def _backward_errors(torch, theta, x, u):
    """Per-layer relative errors (W1, b1, ..., W4, b4) of the library's gradient against the
    quantized oracle network's, and the loss against the oracle's."""
    from paper_2405_04690_gb300 import _lib as L
    B = x.shape[0]
    net = L.Mdn(B)
    L.mdn_set_params(net, torch.from_numpy(theta.astype(np.float32)).cuda())
    grad = torch.zeros(MD.n_params(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    L.mdn_backward(net, xt, torch.from_numpy(u.astype(np.float32)).cuda(), grad, loss)
    L.mdn_status(net)
    net.close()
    got = grad.cpu().numpy().astype(np.float64)
    want = MD.backward(theta, x, u, quantized=True)
    nll = MD.nll(theta, x, u)
    assert abs(loss.item() - nll) < 1e-3 * abs(nll), (loss.item(), nll)
    errs, k = [], 0
    for o, i in MD.LAYERS:
        for n in (o * i, o):
            errs.append(rel_l2(got[k:k + n], want[k:k + n]))
            k += n
    return errs


def test_backward_matches_oracle_layer_by_layer():
    torch = torch_cuda()
    g = np.random.default_rng(7)
    B = 1000
    theta, x, _, _ = _setup(torch, g, B)
    u = g.uniform(0.02, 0.98, (B, MD.N_DIM)).astype(np.float32).astype(np.float64)
    errs = _backward_errors(torch, theta, x, u)
    assert max(errs) < 1e-2, errs


def test_backward_to_1e3_away_from_relu_kinks():
    """Rows whose oracle pre-activations all keep 1e-3 of their RMS away from zero: both
    sides then take the same ReLU branches, and the gradient is held to 1e-3 (a few hundred
    rows: three 128-row tiles, two k-splits of the weight-gradient products)."""
    torch = torch_cuda()
    g = np.random.default_rng(7)
    B = 1000
    theta, x, _, _ = _setup(torch, g, B)
    u = g.uniform(0.02, 0.98, (B, MD.N_DIM)).astype(np.float32).astype(np.float64)
    _, acts = MD.forward(theta, x, quantized=True)
    keep = np.ones(B, bool)
    for li, (w, b) in enumerate(MD.unpack(theta)[:3]):
        z = acts[li] @ MD.to_bf16(w).T + b
        keep &= (np.abs(z) / np.sqrt(np.mean(z * z))).min(axis=1) > 1e-3
    assert 257 <= keep.sum() < B, keep.sum()
    errs = _backward_errors(torch, theta, x[keep], u[keep])
    assert max(errs) < 1e-3, errs


def test_adam_matches_oracle_update():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = np.random.default_rng(8)
    n = MD.n_params()
    p = g.normal(0, 0.05, n).astype(np.float32)
    m = g.normal(0, 1e-3, n).astype(np.float32)
    v = (g.normal(0, 1e-3, n) ** 2).astype(np.float32)
    gr = g.normal(0, 1e-2, n).astype(np.float32)
    step, lr = 5, 1e-3
    wp, wm, wv = MD.adam(p.astype(np.float64), m.astype(np.float64), v.astype(np.float64), gr.astype(np.float64),
                         step, lr)
    net = L.Mdn(16)
    tp, tm, tv = (torch.from_numpy(a.copy()).cuda() for a in (p, m, v))
    L.mdn_adam(net, tp, tm, tv, torch.from_numpy(gr).cuda(), step, lr)
    # float32 arithmetic: 1 - b2 = 0.001 is not exact in float32 (relative 1.3e-5), so v and
    # the update carry ~1e-5 relative error; m = 0.9 m + 0.1 g can cancel, leaving a few ulps
    # of its two terms; p itself adds half an ulp of its magnitude
    np.testing.assert_allclose(tm.cpu().numpy(), wm, rtol=1e-5, atol=2e-9)
    np.testing.assert_allclose(tv.cpu().numpy(), wv, rtol=1e-4, atol=1e-15)
    dp_gpu = tp.cpu().numpy().astype(np.float64) - p
    dp_ora = wp - p
    c1 = 1.0 / (1.0 - 0.9 ** step)
    dm = 4e-7 * (0.9 * np.abs(m) + 0.1 * np.abs(gr))           # m's rounding
    den = np.sqrt(wv / (1.0 - 0.999 ** step)) + 1e-8
    bound = 1e-4 * np.abs(dp_ora) + lr * c1 * dm / den + 2 ** -24 * np.abs(p) + 1e-12
    assert np.all(np.abs(dp_gpu - dp_ora) <= bound), np.max(np.abs(dp_gpu - dp_ora) / bound)
    net.close()


def _task(g, n):
    """Learnable synthetic task: u's first coordinates are functions of the features."""
    x = _bf16(g.normal(0, 1, (n, MD.N_IN)))
    u = np.empty((n, MD.N_DIM))
    u[:, 0] = 1 / (1 + np.exp(-x[:, 0] - 0.5 * x[:, 1]))
    u[:, 1] = 1 / (1 + np.exp(-x[:, 513]))
    u[:, 2:] = g.uniform(0.3, 0.7, (n, MD.N_DIM - 2))
    return x, np.clip(u, 1e-4, 1 - 1e-4)


def test_training_lowers_the_loss_and_is_deterministic():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = np.random.default_rng(9)
    B, steps = 512, 150
    x, u = _task(g, B * 8)
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    theta0 = MD.init_params(np.random.default_rng(10), scale=1.0).astype(np.float32)
    net = L.Mdn(B)
    finals = []
    for rep in range(2):
        p = torch.from_numpy(theta0.copy()).cuda()
        m = torch.zeros_like(p)
        v = torch.zeros_like(p)
        L.mdn_set_params(net, p)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        first = None
        for s in range(1, steps + 1):
            j = (s - 1) % 8
            L.mdn_train_step(net, p, m, v, xt[j * B:(j + 1) * B], ut[j * B:(j + 1) * B], s, 1e-3, loss)
            if s == 1:
                first = loss.item()
        L.mdn_status(net)
        finals.append((first, loss.item(), p.cpu().numpy()))
    (l0, l1, p1), (m0, m1, p2) = finals
    assert np.isfinite(l1) and l1 < l0 - 2.0, (l0, l1)
    assert l0 == m0 and l1 == m1 and np.array_equal(p1, p2)
    # the trained network's density is close to the oracle's at the trained parameters
    raw = torch.zeros((B, MD.N_OUT), dtype=torch.float32, device="cuda")
    L.mdn_forward(net, xt[:B], raw)
    lq_gpu = MD.log_q(raw.cpu().numpy().astype(np.float64), u[:B])
    lq_ora = MD.log_q(MD.forward(p1.astype(np.float64), x[:B], quantized=True)[0], u[:B])
    assert abs(np.mean(lq_gpu) - np.mean(lq_ora)) < 1e-3 * (1 + abs(np.mean(lq_ora)))
    net.close()


def test_train_epoch_equals_single_steps_and_checks_indices():
    # mdn_train_epoch (device gather + steps in one call) = the same minibatches through
    # mdn_train_step, bit for bit; an out-of-range row index is reported, not read.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = np.random.default_rng(19)
    B, n = 96, 500
    x, u = _task(g, n)
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    order = g.permutation(n)[:3 * B].astype(np.int32)
    theta0 = MD.init_params(np.random.default_rng(20)).astype(np.float32)
    net = L.Mdn(B)
    res = []
    for mode in ("steps", "epoch"):
        p = torch.from_numpy(theta0.copy()).cuda()
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        L.mdn_set_params(net, p)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        if mode == "steps":
            for k in range(3):
                idx = torch.from_numpy(order[k * B:(k + 1) * B].astype(np.int64)).cuda()
                L.mdn_train_step(net, p, m, v, xt.index_select(0, idx).contiguous(),
                                 ut.index_select(0, idx).contiguous(), k + 1, 1e-3, loss)
        else:
            L.mdn_train_epoch(net, p, m, v, xt, ut, torch.from_numpy(order).cuda(), B, 0, 1e-3, loss)
        L.mdn_status(net)
        res.append((p.cpu().numpy(), loss.item()))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]
    bad = order[:B].copy()
    bad[5] = n + 3
    p = torch.from_numpy(theta0.copy()).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    L.mdn_train_epoch(net, p, m, v, xt, ut, torch.from_numpy(bad).cuda(), B, 0, 1e-3)
    with pytest.raises(L.GbkError) as ei:
        L.mdn_status(net)
    assert ei.value.status == 2
    net.close()


def _raw_rows(g, n):
    from test_oracle_mdn import raw_from
    rows = []
    for _ in range(n):
        pi = g.dirichlet(np.ones(MD.N_COMP))
        mu = g.uniform(0.05, 0.95, (MD.N_COMP, MD.N_DIM))
        s = np.exp(g.uniform(-6, -0.5, (MD.N_COMP, MD.N_DIM)))
        rows.append(raw_from(pi, mu, s))
    return np.asarray(rows).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec,tol_u,tol_lq", [("fp64", 1e-12, 1e-11), ("mixed", 2e-5, 2e-4)])
def test_mixture_draws_and_densities_match_oracle(prec, tol_u, tol_lq):
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = np.random.default_rng(21)
    n, eps = 400, 0.15
    raw = _raw_rows(g, n)
    words = g.integers(0, 2 ** 32, (n, 9), dtype=np.uint64)
    rt = torch.from_numpy(raw.astype(np.float32)).cuda()
    wt = torch.from_numpy(words.astype(np.uint32).view(np.int32)).cuda()
    u = torch.zeros((n, MD.N_DIM), dtype=torch.float32, device="cuda")
    lq = torch.zeros(n, dtype=torch.float32, device="cuda")
    L.mdn_sample_logpdf(rt, eps, L.PRECISION[prec], words=wt, u_out=u, logq=lq)
    ug = u.cpu().numpy().astype(np.float64)
    uo = np.array([MD.draw_unit(raw[i], int(words[i, 0]), [int(w) for w in words[i, 1:]]) for i in range(n)])
    # u_out is float32: compare at float32 resolution in FP64 mode
    tu = max(tol_u, 2 ** -24)
    assert np.max(np.abs(ug - uo)) < tu * 4, np.max(np.abs(ug - uo))
    # densities at given points (float32 points, so both sides evaluate the same u)
    pts = g.uniform(0, 1, (n, MD.N_DIM)).astype(np.float32)
    L.mdn_sample_logpdf(rt, eps, L.PRECISION[prec], u_in=torch.from_numpy(pts).cuda(), logq=lq)
    want = np.array([MD.log_q_defensive(raw[i], pts[i].astype(np.float64), eps) for i in range(n)])
    got = lq.cpu().numpy().astype(np.float64)
    # logq is returned as float32
    assert np.max(np.abs(got - want) / (1 + np.abs(want))) < max(tol_lq, 2 ** -22), np.max(np.abs(got - want))
