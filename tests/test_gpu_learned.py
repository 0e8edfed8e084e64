"""The learned warm start through the C ABI: gradients and Adam against the FP64 network
reference, and the gain of the trained network over the zero start on held-out systems."""

import numpy as np
import pytest

from oracle import mlp_oracle as MO
from paper_1910_11505_gb300 import learned, sg, workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11505_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


def _unflatten(flat, dims):
    i, h1, h2, d = dims
    shapes = [(h1, i), (h1,), (h2, h1), (h2,), (d, h2), (d,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(flat[o:o + n].astype(np.float64).reshape(s))
        o += n
    return out


def _bf16_round(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_matches_reference(bf16):
    dims = (6, 16, 8, 40)
    net = sg.SGNet(*dims, max_batch=16, bf16=bf16, seed=3)
    rng = np.random.default_rng(0)
    flat = rng.normal(scale=0.4, size=net.num_params).astype(np.float32)
    net.set(0, flat)
    stats = np.concatenate([rng.normal(size=6), 0.5 + rng.random(6)]).astype(np.float32)
    net.set(2, stats)
    Z = rng.normal(size=(7, 6)).astype(np.float32)
    T = rng.normal(size=(7, 40)).astype(np.float32)
    loss = net.loss_grad(torch.from_numpy(Z).cuda(), torch.from_numpy(T).cuda())
    grad = net.get(1).astype(np.float64)
    params = _unflatten(flat, dims)
    if bf16:  # the output layer computes from the BF16 copy of W3
        params[4] = _bf16_round(params[4])
    ref_loss, ref = MO.loss_and_grads(params, Z.astype(np.float64), T.astype(np.float64),
                                      stats[:6].astype(np.float64), stats[6:].astype(np.float64))
    ref_flat = np.concatenate([g.ravel() for g in ref])
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    err = np.abs(grad - ref_flat).max() / np.abs(ref_flat).max()
    assert err <= 2e-5, err
    net.close()


def test_adam_step_matches_reference():
    dims = (6, 16, 8, 40)
    net = sg.SGNet(*dims, max_batch=16, bf16=False, seed=4)
    rng = np.random.default_rng(1)
    Z = rng.normal(size=(5, 6)).astype(np.float32)
    T = rng.normal(size=(5, 40)).astype(np.float32)
    p0 = net.get(0).astype(np.float64)
    st = net.get(2).astype(np.float64)
    params = _unflatten(p0.astype(np.float32), dims)
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    small = None
    for t in (1, 2):
        net.loss_grad(torch.from_numpy(Z).cuda(), torch.from_numpy(T).cuda(), want_loss=False)
        net.adam_step(1e-2)
        _, g = MO.loss_and_grads(params, Z.astype(np.float64), T.astype(np.float64), st[:6], st[6:])
        gf = np.abs(np.concatenate([x.ravel() for x in g]))
        small = gf < 1e-5 if small is None else small | (gf < 1e-5)
        params = MO.adam_step(params, g, m, v, t, 1e-2)
    got = net.get(0).astype(np.float64)
    ref = np.concatenate([p.ravel() for p in params])
    # an Adam step is lr * g / (|g| + eps): where |g| is near rounding level its direction is
    # not fixed by the arithmetic, so those parameters are excluded
    assert small.mean() < 0.05
    assert np.abs(got - ref)[~small].max() <= 1e-5
    net.close()


def test_predict_equals_forward():
    net = sg.SGNet(6, 16, 8, 40, max_batch=16, bf16=True, seed=5)
    Z = torch.randn(9, 6, device="cuda")
    Y = torch.empty(9, 40, device="cuda")
    X = torch.empty(9, 40, dtype=torch.float64, device="cuda")
    net.forward(Z, Y)
    net.predict(Z, X)
    torch.cuda.synchronize()
    assert torch.equal(X.float(), Y)
    net.close()


def _hidden_ref(params, Z, stats):
    """h2 of the network in FP64 for inputs Z (the layers before the output layer)."""
    W1, b1, W2, b2 = params[:4]
    zh = (Z.astype(np.float64) - stats[:6]) / stats[6:]
    return np.tanh(np.tanh(zh @ W1.T + b1) @ W2.T + b2)


@pytest.mark.parametrize("h2,out,B", [(64, 300, 200), (40, 128, 129), (64, 1000, 7)])
def test_tensor_core_output_layer_matches_reference(h2, out, B):
    # with a BF16 copy of W3 the output layer runs as tcgen05 MMAs on BF16 operands (h2 and W3
    # rounded to BF16) with FP32 accumulation; sizes cover ragged batch and unit tiles and
    # h2 < 64 (K zero-padded)
    dims = (6, 16, h2, out)
    net = sg.SGNet(*dims, max_batch=256, bf16=True, seed=21)
    rng = np.random.default_rng(5)
    flat = rng.normal(scale=0.4, size=net.num_params).astype(np.float32)
    net.set(0, flat)
    stats = np.concatenate([rng.normal(size=6), 0.5 + rng.random(6)]).astype(np.float32)
    net.set(2, stats)
    Z = rng.normal(size=(B, 6)).astype(np.float32)
    Y = torch.empty(B, out, device="cuda")
    net.forward(torch.from_numpy(Z).cuda(), Y)
    params = _unflatten(flat, dims)
    W3b, b3 = _bf16_round(params[4]), params[5]
    hb = _bf16_round(_hidden_ref(params, Z, stats.astype(np.float64)))
    ref = hb @ W3b.T + b3
    # the GPU's FP32 hidden layers may round an h2 value to the neighbouring BF16 number (one
    # unit 2^-8 of it) where the FP64 one falls the other side; FP32 accumulation of 64 terms
    terms = np.abs(hb)[:, None, :] * np.abs(W3b)[None, :, :]
    bound = 2.0 ** -8 * terms.max(axis=2) + 64 * 2.0 ** -24 * terms.sum(axis=2) + 1e-7
    got = Y.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound), np.abs(got - ref).max()
    # the fixed-output-layer training loss (residual epilogue of the same kernel) equals the
    # mean square of the forward result against the targets
    T = rng.normal(size=(B, out)).astype(np.float32)
    net.set_basis(torch.from_numpy(T).cuda())
    Y2 = torch.empty(B, out, device="cuda")
    net.forward(torch.from_numpy(Z).cuda(), Y2)
    loss = net.loss_grad(torch.from_numpy(Z).cuda(), torch.from_numpy(T).cuda())
    want = float(((Y2.double().cpu().numpy() - T) ** 2).mean())
    assert abs(loss - want) <= 1e-5 * want
    net.close()


@pytest.mark.parametrize("B,out", [(200, 300), (129, 1000), (7, 64)])
def test_tensor_core_backprop_matches_reference(B, out):
    # with the output layer fixed and a BF16 copy of W3, a training step runs the output layer
    # and dH2 = dY W3 (split over the units, K padded to a multiple of 64) as tcgen05 MMAs on
    # BF16 dY and W3; the hidden layers' gradient then follows in FP32.  Reference: dY formed
    # from the tensor-core forward result exactly as the kernel rounds it (FP32 residual and
    # scale, BF16), then back-propagated in FP64.
    dims = (6, 16, 64, out)
    net = sg.SGNet(*dims, max_batch=256, bf16=True, seed=23)
    rng = np.random.default_rng(6)
    flat = rng.normal(scale=0.4, size=net.num_params).astype(np.float32)
    net.set(0, flat)
    stats = np.concatenate([rng.normal(size=6), 0.5 + rng.random(6)]).astype(np.float32)
    net.set(2, stats)
    Z = rng.normal(size=(B, 6)).astype(np.float32)
    T = rng.normal(size=(B, out)).astype(np.float32)
    net.set_basis(torch.from_numpy(T).cuda())
    Y = torch.empty(B, out, device="cuda")
    net.forward(torch.from_numpy(Z).cuda(), Y)
    net.loss_grad(torch.from_numpy(Z).cuda(), torch.from_numpy(T).cuda())
    grad = net.get(1).astype(np.float64)
    params = _unflatten(net.get(0), dims)
    W1, b1, W2, b2, W3 = params[:5]
    scale = np.float32(2.0) / (np.float32(B) * np.float32(out))
    dY = _bf16_round(scale * (Y.cpu().numpy() - T))
    dH2 = dY @ _bf16_round(W3)
    zh = (Z.astype(np.float64) - stats[:6]) / stats[6:]
    H1 = np.tanh(zh @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    dA2 = dH2 * (1.0 - H2 * H2)
    dA1 = (dA2 @ W2) * (1.0 - H1 * H1)
    ref = np.concatenate([(dA1.T @ zh).ravel(), dA1.sum(0), (dA2.T @ H1).ravel(), dA2.sum(0)])
    got = grad[:ref.size]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-4, err
    net.close()


def test_trained_network_reduces_gmres_iterations():
    # small mesh: n = 16, M = 2, p = 2 (D = 289 x 6); sigma ~ U[0.1, 1.5], ell ~ U[0.25, 2]
    draws = W.c5_draws(288, seed=11)
    base = dict(n=16, M=2, p=2, precond="mean")
    train_p = [dict(base, sigma=s, ell=l) for s, l in draws[:256]]
    test_p = [dict(base, sigma=s, ell=l) for s, l in draws[256:288]]
    Z, T, gen = learned.generate(train_p, chunk=64)
    net = sg.SGNet(Z.shape[1], 64, 64, T.shape[1], max_batch=64, bf16=True, seed=9)
    net.set_stats(Z, T)
    net.set_basis(T)
    learned.train(net, Z, T, steps=4000, batch=64, lr=2e-3)
    ev = learned.warm_start_eval(net, test_p)
    assert ev["rc"] == (sg.SG_OK, sg.SG_OK)
    assert max(ev["warm_resid"]) <= 1e-8  # the final FP64 residual still decides
    zero, warm = np.array(ev["zero_iters"]), np.array(ev["warm_iters"])
    assert warm.mean() < 0.9 * zero.mean(), ev
    assert (warm <= zero).mean() >= 0.75, ev
    net.close()


def test_output_basis_is_orthogonal_and_fixed_by_adam():
    # the output layer spans the centred training targets (scaled orthonormal columns) and Adam
    # leaves it unchanged while the hidden layers train
    rng = np.random.default_rng(7)
    D = 300
    T = torch.from_numpy(rng.normal(size=(24, D)).astype(np.float32)).cuda()
    Z = torch.from_numpy(rng.normal(size=(24, 6)).astype(np.float32)).cuda()
    net = sg.SGNet(6, 16, 8, D, max_batch=32, bf16=False, seed=2)
    net.set_stats(Z, T)
    net.set_basis(T)
    p0 = net.get(0).astype(np.float64)
    dims = (6, 16, 8, D)
    W3 = _unflatten(p0.astype(np.float32), dims)[4]
    g = W3.T @ W3
    assert np.abs(g - np.diag(np.diag(g))).max() <= 1e-5 * np.diag(g).max()
    Tc = T.cpu().numpy().astype(np.float64) - T.cpu().numpy().astype(np.float64).mean(0)
    # the first 8 centred targets lie in the span of the columns
    Q = W3 / np.linalg.norm(W3, axis=0)
    resid = Tc[:8].T - Q @ (Q.T @ Tc[:8].T)
    assert np.abs(resid).max() <= 1e-4 * np.abs(Tc).max()
    net.train_step(Z[:16], T[:16], 1e-2)
    p1 = net.get(0).astype(np.float64)
    nsmall = 16 * 6 + 16 + 8 * 16 + 8
    assert np.array_equal(p1[nsmall:], p0[nsmall:])
    assert not np.array_equal(p1[:nsmall], p0[:nsmall])
    net.close()
