"""Warm-start network: kernels against the FP64 reference, and the gain over
rest starts.  The network, its backward pass and Adam run in the library's
CUDA kernels; the reference is oracle/surrogate.py (float64, autograd)."""
import numpy as np
import pytest

from paper_1801_04577_gb300 import inputs as I
from paper_1801_04577_gb300 import surrogate as SG
from paper_1801_04577_gb300.net import Net, layer_shapes, weights_as_used

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _batch(G, cin, cout, N, seed):
    r = I.splitmix64_uniform(seed, N * (cin + cout + 1) * G * G)
    o = N * cin * G * G
    x = (2 * r[:o] - 1).reshape(N, cin, G, G).astype(np.float32)
    t = (2 * r[o:o + N * cout * G * G] - 1).reshape(N, cout, G, G).astype(np.float32)
    m = (r[o + N * cout * G * G:] > 0.25).reshape(N, G, G).astype(np.float32)
    return x, t, m


@pytest.mark.parametrize("G,base,levels,N", [(16, 4, 3, 2), (64, 24, 4, 2)])
def test_net_forward_and_gradients_match_reference(G, base, levels, N):
    from oracle import surrogate as S
    net = Net(G, 5, 3, base, levels, N, seed=3)
    x, t, m = _batch(G, 5, 3, N, seed=G + base)
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, m))
    y = torch.empty((N, 3, G, G), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    loss, g = net.gradients(xd, td, md)
    shapes = layer_shapes(G, 5, 3, base, levels)
    p = weights_as_used(net.get_params(), shapes)
    L_ref, g_ref, y_ref = S.loss_and_grad(p.astype(np.float64), shapes, levels, x, t, m)
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    assert np.abs(yg - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    assert loss == pytest.approx(L_ref, rel=1e-5)
    # per layer: max-norm relative error of the weight and bias gradients
    off = 0
    for ci, co, k in shapes:
        for n in (co * ci * k * k, co):
            a, b = g[off:off + n], g_ref[off:off + n]
            assert np.abs(a - b).max() <= 1e-4 * max(np.abs(b).max(), 1e-12), (ci, co, k, n)
            off += n
    net.close()


def test_adam_training_reduces_loss_on_fixed_batch():
    G, N = 16, 4
    net = Net(G, 5, 3, 8, 3, N, seed=5)
    x, t, m = _batch(G, 5, 3, N, seed=77)
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, m))
    first = net.train_step(xd, td, md, 3e-3)
    for _ in range(60):
        last = net.train_step(xd, td, md, 3e-3)
    assert last < 0.5 * first
    net.close()


def test_warm_start_reaches_steady_state_in_fewer_steps():
    """Train on solver-generated steady states of 32^2 obstacle cavities, then
    solve held-out problems from rest and from the network's prediction: the
    warm start needs fewer steps to reach the residual tolerance, and both
    starts converge to the same Nusselt number."""
    G, tol, cap = 32, 1e-6, 30000
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    train_ws = I.obstacle_cavities(384, G, seed=101)
    Y, conv, _ = SG.generate(train_ws, tol, cap, stream=stream.cuda_stream)
    X = SG.encode(train_ws)
    M = X[:, 0].copy()
    net = SG.make_net(G, base=16, levels=3, max_batch=32, seed=9, stream=stream.cuda_stream)
    Xd, Yd, Md = (torch.from_numpy(a).cuda() for a in (X, Y, M))
    losses = SG.train(net, Xd, Yd, Md, epochs=60, batch=32, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    test_ws = I.obstacle_cavities(32, G, seed=9001)
    r = SG.compare_starts(net, test_ws, tol, cap, stream=stream.cuda_stream)
    both = (r["rest_steps"] > 0) & (r["warm_steps"] > 0)
    assert both.sum() >= 24
    rest, warm = r["rest_steps"][both], r["warm_steps"][both]
    assert np.median(warm) < 0.8 * np.median(rest), (np.median(warm), np.median(rest))
    nu_rel = np.abs(r["nu_warm"] - r["nu_rest"])[both] / np.abs(r["nu_rest"][both])
    assert np.median(nu_rel) < 2e-2
    net.close()
