"""GPU network kernels against the float64 network of oracle/cnn.py.

Features are compared on simulated stacks; the forward activations, the
outputs and every parameter gradient are compared on the same BF16-rounded
weights and features (the network computes with BF16 layer inputs and FP32
accumulation, so the bar is a relative L2 error of a few BF16 roundings);
the AdamW step is compared with its formula in float32.
"""
import numpy as np
import pytest

from oracle import cnn
from paper_2407_20469_gb300 import apic, learn, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_20469_gb300 import build
    build.build()
    return apic.load()


def _stacks(n, count, seed, blank_frac=0.3):
    plan = apic.Plan.from_illumination(n, synth.illumination(), max_tiles=max(count, 1))
    uv, zern, blank = learn.draw_tiles(count, seed, learn.field_table(), blank_frac)
    I = learn.simulate(plan, zern, blank, seed)
    return plan, I, uv, zern, blank


@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_features_match_definition(lib, n):
    plan, I, uv, zern, blank = _stacks(n, 3, 40 + n)
    feat = torch.empty((3, 64, 64, 8), dtype=torch.float32, device="cuda")
    plan.features(3, I, feat)
    got = feat.cpu().numpy().transpose(0, 3, 1, 2)
    Ih = I.cpu().numpy().astype(np.float64)
    for t in range(3):
        ref = cnn.features(Ih[t, :8])
        err = np.abs(got[t] - ref)
        print(f"n={n} tile {t}: max |df| {err.max():.2e}, mean {err.mean():.2e}")
        assert err.max() < 5e-3 and err.mean() < 2e-4


def test_features_reject_unsupported_plans(lib):
    """The network takes exactly 8 NA-matching images: a 12 + 22 plan is refused."""
    plan = apic.Plan.from_illumination(64, synth.illumination_12_22(), max_tiles=1, upsample=3)
    x = torch.zeros((1, 34, 64, 64), device="cuda")
    f = torch.zeros((1, 64, 64, 8), device="cuda")
    with pytest.raises(apic.ApicError):
        plan.features(1, x, f)


@pytest.fixture(scope="module")
def case(lib):
    """Small batch: real features, random positions, BF16-rounded weights."""
    plan, I, uv, zern, blank = _stacks(64, 3, 7)
    feat = torch.empty((3, 64, 64, 8), dtype=torch.float32, device="cuda")
    plan.features(3, I, feat)
    flat = bf16(learn.init_params(3)).astype(np.float32)
    # non-zero biases so that their paths are exercised
    p = apic.unpack_params(flat)
    rng = np.random.default_rng(5)
    for l in range(6):
        p[f"b{l}"] = bf16(rng.normal(0, 0.05, p[f"b{l}"].shape))
    flat = apic.pack_params(p)
    p = apic.unpack_params(flat)
    x = bf16(feat.cpu().numpy()).transpose(0, 3, 1, 2)
    target = rng.uniform(-1, 1, (3, 15)).astype(np.float32)
    target[:, :3] = 0
    return dict(feat=feat, uv=uv, flat=flat, p=p, x=x, target=target)


def test_forward_matches_oracle(case):
    B = 3
    net = apic.Net(4)
    net.set_params(case["flat"])
    uv = torch.as_tensor(case["uv"], device="cuda")
    out = torch.empty((B, 15), dtype=torch.float32, device="cuda")
    net.forward(B, case["feat"], uv, out)
    y_ref, (cache, h_in, z4, h4) = cnn.forward(case["p"], case["x"], case["uv"].astype(np.float64))
    for l in range(4):
        r_ref = np.maximum(cache[l][1], 0).transpose(0, 2, 3, 1)
        e = rel(net.activation(l, B), r_ref)
        print(f"conv {l}: rel L2 {e:.2e}")
        assert e < 2e-2
    e_h = rel(net.activation(4, B), h_in)
    e_4 = rel(net.activation(5, B), h4)
    o = out.cpu().numpy()
    e_y = rel(o[:, 3:], y_ref)
    print(f"dense in {e_h:.2e}, hidden {e_4:.2e}, outputs {e_y:.2e}")
    assert e_h < 2e-2 and e_4 < 3e-2 and e_y < 3e-2
    assert np.all(o[:, :3] == 0)


def test_gradients_match_oracle(case):
    B = 3
    net = apic.Net(4)
    net.set_params(case["flat"])
    uv = torch.as_tensor(case["uv"], device="cuda")
    net.forward(B, case["feat"], uv)
    tgt = torch.as_tensor(case["target"], device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.backward(tgt, loss)
    g = apic.unpack_params(net.get_grads())
    loss_ref, g_ref = cnn.loss_and_grads(case["p"], case["x"], case["uv"].astype(np.float64),
                                         case["target"][:, 3:].astype(np.float64))
    print(f"loss {loss.item():.6f} vs {loss_ref:.6f}")
    assert abs(loss.item() - loss_ref) <= 2e-2 * loss_ref
    for name, _ in apic.param_shapes():
        e = rel(g[name], g_ref[name])
        print(f"d{name}: rel L2 {e:.2e}")
        assert e < 5e-2, name


def test_adamw_step_matches_formula(case):
    B = 3
    net = apic.Net(4)
    net.set_params(case["flat"])
    uv = torch.as_tensor(case["uv"], device="cuda")
    tgt = torch.as_tensor(case["target"], device="cuda")
    p0 = net.get_params().astype(np.float64)
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 1e-2
    for step in (1, 2):
        net.forward(B, case["feat"], uv)
        net.backward(tgt)
        g = net.get_grads().astype(np.float64)
        net.adamw(lr, step, b1, b2, eps, wd)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p0 = p0 - lr * ((m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps) + wd * p0)
        p1 = net.get_params().astype(np.float64)
        assert np.max(np.abs(p1 - p0)) < 1e-6
        p0 = p1


def test_network_rejects_bad_arguments(lib):
    net = apic.Net(2)
    f = torch.zeros((3, 64, 64, 8), device="cuda")
    with pytest.raises(apic.ApicError):
        net.forward(3, f, None)
    with pytest.raises(apic.ApicError):
        net.set_params(np.zeros(10, np.float32))
    fresh = apic.Net(1)
    with pytest.raises(apic.ApicError):
        fresh.backward(torch.zeros((1, 15), device="cuda"))


def test_checkpoint_blob_round_trip_through_the_c_abi(lib):
    """A BF16 checkpoint written by learn.bf16_blob and read by apic_net_load gives the
    network exactly the BF16-rounded parameters, and the same forward pass as setting
    those values directly."""
    from paper_2407_20469_gb300 import learn
    rng = np.random.default_rng(17)
    p = apic.pack_params(cnn.init_params(rng)) + rng.standard_normal(459244).astype(np.float32) * 1e-3
    a, b = apic.Net(4), apic.Net(4)
    a.load_blob(learn.bf16_blob(p))
    got = a.get_params()
    assert np.array_equal(got, learn.bf16_values(p))
    b.set_params(learn.bf16_values(p))
    feat = torch.randn((4, 64, 64, 8), device="cuda")
    uv = torch.rand((4, 2), device="cuda") * 2 - 1
    oa = torch.zeros((4, 15), device="cuda")
    ob = torch.ones((4, 15), device="cuda")
    a.forward(4, feat, uv, oa)
    b.forward(4, feat, uv, ob)
    torch.cuda.synchronize()
    assert torch.equal(oa, ob)
    with pytest.raises(apic.ApicError):
        a.load_blob(learn.bf16_blob(p)[:-2])
    a.close()
    b.close()
