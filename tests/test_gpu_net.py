"""GPU checks of the learned correction's kernels against the CPU reference
(oracle/net_oracle.py).  Each layer is fed the GPU's own bfloat16 input, so
the comparison is FP32 accumulation against FP64 plus, for the hidden layers,
the bfloat16 rounding decision of every activation (the GPU's value must be
the bfloat16 neighbour of the exact value on the correct side, i.e. within one
bfloat16 ulp)."""
import numpy as np
import pytest

from oracle import net_oracle as no
from paper_1311_3004_gb300 import fvna
from paper_1311_3004_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    from paper_1311_3004_gb300 import build
    build.build()
    return t


def bits_to_f64(h):
    u = h.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def _setup(torch, B=2, H=20, W=45, seed=0, scale=3.0):
    rng = np.random.default_rng(seed)
    p = no.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.05, size=p[k].shape)
    x = rng.normal(size=(B, 3, H, W)).astype(np.float32)
    net = fvna.Net(fvna.net_params_flat(p))
    xd = torch.from_numpy(x).cuda()
    return p, x, xd, net, scale


def test_forward_layers_match_reference(torch):
    p, x, xd, net, s = _setup(torch)
    y, h1, h2 = net.forward(xd, in_scale=s, hidden=True)
    y = y.cpu().numpy().astype(np.float64)
    h1 = bits_to_f64(h1).transpose(0, 3, 1, 2)
    h2 = bits_to_f64(h2).transpose(0, 3, 1, 2)
    q = no.bf16
    w1, w2, w3 = q(p["w1"]), q(p["w2"]), q(p["w3"])
    for b in range(x.shape[0]):
        x0 = q(x[b].astype(np.float64) * np.float32(s))
        z1 = np.maximum(no.conv3x3(x0, w1, p["b1"].astype(np.float32).astype(np.float64)), 0)
        ulp1 = np.maximum(np.abs(z1), 1e-30) * 2.0 ** -7
        assert np.all(np.abs(h1[b] - z1) <= ulp1 + 1e-6), np.max(np.abs(h1[b] - z1) - ulp1)
        z2 = np.maximum(no.conv3x3(h1[b], w2, p["b2"].astype(np.float32).astype(np.float64)), 0)
        ulp2 = np.maximum(np.abs(z2), 1e-30) * 2.0 ** -7
        assert np.all(np.abs(h2[b] - z2) <= ulp2 + 1e-6)
        yr = no.conv3x3(h2[b], w3, p["b3"].astype(np.float32).astype(np.float64))
        assert np.max(np.abs(y[b] - yr)) <= 1e-5 * (1 + np.max(np.abs(yr)))
        # and almost every rounding decision agrees exactly with the FP64 one
        assert np.mean(h1[b] == q(z1)) > 0.999
    net.close()


def test_backward_matches_reference(torch):
    p, x, xd, net, s = _setup(torch, seed=1)
    y, h1, h2 = net.forward(xd, in_scale=s, hidden=True)
    rng = np.random.default_rng(5)
    gy = rng.normal(size=x.shape).astype(np.float32)
    g = net.backward(xd, torch.from_numpy(gy).cuda(), in_scale=s).cpu().numpy()
    gd = fvna.net_params_dict(g)
    h1 = bits_to_f64(h1).transpose(0, 3, 1, 2)
    h2 = bits_to_f64(h2).transpose(0, 3, 1, 2)
    q = no.bf16
    ref = {k: 0.0 for k in gd}
    for b in range(x.shape[0]):
        x0 = q(x[b].astype(np.float64) * np.float32(s))
        cache = (x0, h1[b], h2[b], q(p["w1"]), q(p["w2"]), q(p["w3"]))
        gb = no.backward(gy[b].astype(np.float64), cache)
        for k in ref:
            ref[k] = ref[k] + gb[k]
    for k in gd:
        err = np.max(np.abs(gd[k] - ref[k])) / (np.max(np.abs(ref[k])) + 1e-30)
        assert err < 1e-4, (k, err)
    net.close()


def test_training_reduces_loss(torch):
    """Learn a fixed linear map of the input (reachable by the network)."""
    rng = np.random.default_rng(2)
    net = fvna.Net(fvna.net_params_flat(no.init_params(7)))
    x = torch.from_numpy(rng.normal(size=(8, 3, 32, 32)).astype(np.float32)).cuda()
    t = torch.roll(x, 1, dims=1) * 0.5
    losses = [net.train_step(x, t, 2e-3) for _ in range(300)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    net.close()


def test_correction_hook_in_solver(torch):
    """A network whose only nonzero parameter is b3 adds out_scale * b3 to the
    state after every step; an all-zero network changes nothing."""
    n = 64
    q0 = wl.random_smooth(n, n, 1e-4, seed=3)
    cfg = fvna.make_config(precision=fvna.FP32_PERT, beta=3.5, delta=1e-3, dx=1.0 / 32,
                           dt_fixed=0.01)
    dom = fvna.make_domain(n, n, bc=(fvna.BC_PERIODIC,) * 4)
    s0 = fvna.Solver(cfg, [dom], [q0])
    s0.run(max_steps=5)
    base = s0.q(0)
    s0.close()
    flat = np.zeros(fvna.NET_PARAMS, dtype=np.float32)
    zero = fvna.Net(flat)
    s1 = fvna.Solver(cfg, [dom], [q0])
    s1.set_correction(zero, 1e3, 1e-4)
    s1.run(max_steps=5)
    assert np.array_equal(s1.q(0), base)
    s1.close()
    flat[-3:] = [1.0, -2.0, 0.5]
    bias = fvna.Net(flat)
    s2 = fvna.Solver(cfg, [dom], [q0])
    s2.set_correction(bias, 1e3, 1e-6)
    s2.run(max_steps=5)
    d = s2.q(0) - base
    # a uniform shift does not change the fluxes: the offsets add up exactly
    assert np.allclose(d[0], 5e-6, rtol=1e-3) and np.allclose(d[1], -10e-6, rtol=1e-3)
    assert np.allclose(d[2], 2.5e-6, rtol=1e-3)
    s2.close()
