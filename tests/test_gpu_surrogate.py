"""Warm-start network: kernels against the FP64 reference, and the gain over
rest starts.  The network, its backward pass and Adam run in the library's
CUDA kernels; the reference is oracle/surrogate.py (float64, autograd).

Tolerances.  FP32 CUDA-core convolutions: forward 1e-5, gradients 1e-4
(max-norm relative), FP32 rounding only.  Tensor-core convolutions (both GEMM
operands rounded to bfloat16): against the reference with the same roundings
(rnd=bf16) the results are identical whenever every GEMM sum is exact in FP32
(sparse dyadic weights: forward bit-exact, gradients to FP32 accumulation);
with dense random weights the FP32-vs-FP64 difference of a sum flips an
occasional bfloat16 rounding and the flips spread through the 19 layers, so
the two agree only to the size of the bfloat16 noise itself: sqrt(2 x 19)
roundings of 2^-8 relative give ~2.4e-2, bounded here by 2e-2 (forward, max
relative to max |y|) and 5e-2 (per-layer gradients)."""
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


def _layer_errors(g, g_ref, shapes):
    """max-norm relative error of every layer's weight and bias gradients"""
    out, off = [], 0
    for ci, co, k in shapes:
        for n in (co * ci * k * k, co):
            a, b = g[off:off + n], g_ref[off:off + n]
            out.append(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))
            off += n
    return np.array(out)


@pytest.mark.parametrize("G,base,levels,N", [(16, 4, 3, 2), (64, 24, 4, 2)])
def test_net_forward_and_gradients_match_reference(G, base, levels, N):
    """FP32 CUDA-core convolutions against the float64 reference."""
    from oracle import surrogate as S
    net = Net(G, 5, 3, base, levels, N, seed=3, math="fp32")
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


def _sparse_dyadic_params(shapes, seed, nnz=4):
    """Weights k/8 (k = +-1..4) on about nnz taps per output, biases j/16:
    every GEMM sum of the network then holds few terms of short significands
    and is exact in FP32 as well as in FP64."""
    out = []
    for li, (ci, co, k) in enumerate(shapes):
        K = ci * k * k
        r = I.splitmix64_uniform(seed + li, co * K * 2 + co)
        keep = r[:co * K] < nnz / K
        val = np.floor(r[co * K:2 * co * K] * 8) - 4
        val[val >= 0] += 1
        out.append(np.where(keep, val / 8.0, 0.0))
        out.append(np.floor(r[2 * co * K:] * 8 - 4) / 16.0)
    return np.concatenate(out).astype(np.float32)


@pytest.mark.parametrize("G,base,levels,N", [(64, 24, 4, 2), (16, 48, 3, 2)])
def test_tensor_core_net_exact_when_sums_are_exact(G, base, levels, N):
    """tcgen05 path against the reference with bfloat16-rounded GEMM operands,
    on a problem whose every sum is exact: the forward pass is bit-identical.
    (64^2, widths 24..192: 1.1 M parameters, K up to 2592; widths 48..192:
    input-gradient GEMMs with 288 columns in two tiles.)"""
    from oracle import surrogate as S
    cin, cout = 5, 4  # out_ch 4: the loss normalisation N G^2 4 is a power of two
    shapes = layer_shapes(G, cin, cout, base, levels)
    net = Net(G, cin, cout, base, levels, N, seed=3, math="tensor")
    p = _sparse_dyadic_params(shapes, 100 + G + base)
    net.set_params(p)
    r = I.splitmix64_uniform(7, N * (cin + cout) * G * G)
    x = (np.floor(r[:N * cin * G * G] * 9 - 4) / 4).reshape(N, cin, G, G).astype(np.float32)
    t = (np.floor(r[N * cin * G * G:] * 9 - 4) / 4).reshape(N, cout, G, G).astype(np.float32)
    xd, td = (torch.from_numpy(a).cuda() for a in (x, t))
    y = torch.empty((N, cout, G, G), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    loss, g = net.gradients(xd, td, None)
    assert (weights_as_used(net.get_params(), shapes) == p).all()
    L_ref, g_ref, y_ref = S.loss_and_grad(p.astype(np.float64), shapes, levels, x, t, None, rnd=S.bf16)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), y_ref.astype(np.float32))
    assert loss == pytest.approx(L_ref, rel=1e-12)
    e = _layer_errors(g, g_ref, shapes)
    assert e.max() <= 5e-5, e
    net.close()


@pytest.mark.parametrize("G,base,levels,N", [(16, 4, 3, 2), (64, 24, 4, 2)])
def test_tensor_core_net_matches_bf16_reference(G, base, levels, N):
    """tcgen05 path with dense random weights against the reference with the
    same bfloat16 roundings, within the bfloat16 noise (module docstring)."""
    from oracle import surrogate as S
    net = Net(G, 5, 3, base, levels, N, seed=3, math="tensor")
    x, t, m = _batch(G, 5, 3, N, seed=G + base)
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, m))
    y = torch.empty((N, 3, G, G), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    loss, g = net.gradients(xd, td, md)
    shapes = layer_shapes(G, 5, 3, base, levels)
    p = weights_as_used(net.get_params(), shapes)
    L_ref, g_ref, y_ref = S.loss_and_grad(p.astype(np.float64), shapes, levels, x, t, m, rnd=S.bf16)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - y_ref).max() <= 2e-2 * np.abs(y_ref).max()
    assert loss == pytest.approx(L_ref, rel=1e-3)
    e = _layer_errors(g, g_ref, shapes)
    assert e.max() <= 5e-2, e
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


@pytest.mark.parametrize("math", ["tensor", "fp32"])
def test_replayed_passes_follow_the_buffer_contents(math):
    """The forward and gradient passes are captured on their first call with a
    batch size and replayed afterwards, the caller's tensors copied in and out
    around them: a replay follows new contents of the same tensors and other
    tensors alike, and gives what a first call gives (a fresh network with the
    same weights), bit for bit."""
    G, N = 16, 3
    x, t, m = _batch(G, 5, 3, N, seed=91)
    x2, t2, _ = _batch(G, 5, 3, N, seed=92)
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, m))
    net = Net(G, 5, 3, 8, 3, N, seed=7, math=math)
    l1, g1 = net.gradients(xd, td, md)
    l1b, g1b = net.gradients(xd, td, md)  # replay, same contents
    assert l1b == l1 and np.array_equal(g1b, g1)
    xd.copy_(torch.from_numpy(x2))
    td.copy_(torch.from_numpy(t2))
    torch.cuda.synchronize()  # the network runs on its own stream
    l2, g2 = net.gradients(xd, td, md)  # replay, new contents
    y = torch.empty((N, 3, G, G), device="cuda")
    net.forward(xd, y)
    net.forward(xd, y)
    torch.cuda.synchronize()
    fresh = Net(G, 5, 3, 8, 3, N, seed=7, math=math)
    x2d, t2d = torch.from_numpy(x2).cuda(), torch.from_numpy(t2).cuda()
    l2r, g2r = fresh.gradients(x2d, t2d, md)
    y2 = torch.empty_like(y)
    fresh.forward(x2d, y2)
    torch.cuda.synchronize()
    assert l2 == l2r and np.array_equal(g2, g2r) and l2 != l1
    assert torch.equal(y, y2)
    l3, g3 = net.gradients(x2d, t2d, md)  # replay from other tensors
    assert l3 == l2r and np.array_equal(g3, g2r)
    l4, g4 = net.gradients(x2d, t2d)  # no mask: its own capture
    l4r, g4r = fresh.gradients(x2d, t2d)
    assert l4 == l4r and np.array_equal(g4, g4r) and l4 != l3
    net.close()
    fresh.close()


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
    # the learning rate decays to 2e-4: at a constant 2e-3 the last epochs are
    # noisy and the step saving swings between 10 % and 35 % with the rounding
    # order of the gradient sums
    losses = SG.train(net, Xd, Yd, Md, epochs=60, batch=32, lr=2e-3, lr_final=2e-4)
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
