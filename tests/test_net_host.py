"""CPU checks of the network's parameter layout (no GPU calls)."""
import numpy as np
import pytest

from oracle import cnn
from paper_2407_20469_gb300 import apic


def test_param_count_matches_definition():
    p = cnn.init_params(np.random.default_rng(0))
    assert apic.load().apic_net_param_count() == cnn.param_count(p) == 459244
    assert apic.load().apic_net_feature_count() == 64 * 64 * 8


def test_pack_unpack_round_trip_and_layout():
    rng = np.random.default_rng(1)
    p = cnn.init_params(rng)
    for k in list(p):
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape)
    flat = apic.pack_params(p)
    assert flat.dtype == np.float32 and flat.size == cnn.param_count(p)
    q = apic.unpack_params(flat)
    for k in p:
        assert q[k].shape == p[k].shape
        np.testing.assert_allclose(q[k], p[k].astype(np.float32), rtol=0, atol=0)
    # conv 0: row co has 9 * 8 taps ordered (dy, dx, ci), then the bias
    co, ci, dy, dx = 3, 5, 2, 1
    assert flat[co * 73 + (dy * 3 + dx) * 8 + ci] == np.float32(p["w0"][co, ci, dy, dx])
    assert flat[co * 73 + 72] == np.float32(p["b0"][co])
    # last layer: 12 rows of 256 weights + bias at the end of the vector
    assert flat[-1] == np.float32(p["b5"][11])
    assert flat[-2] == np.float32(p["w5"][11, 255])


def test_parameter_file_round_trip_and_refusals(tmp_path):
    from paper_2407_20469_gb300 import learn
    flat = learn.init_params(7)
    path = str(tmp_path / "net.bin")
    learn.save_params(path, flat, {"epochs": 4, "loss": 0.01})
    got, meta = learn.load_params(path)
    assert got.dtype == np.float32 and np.array_equal(got, flat) and meta == {"epochs": 4, "loss": 0.01}
    raw = open(path, "rb").read()
    open(path, "wb").write(raw[:-4])                       # truncated
    with pytest.raises(ValueError, match="expected"):
        learn.load_params(path)
    open(path, "wb").write(b"NOTANET1" + raw[8:])
    with pytest.raises(ValueError, match="not a network"):
        learn.load_params(path)
    open(path, "wb").write(raw.replace(b'"count": 459244', b'"count": 459243'))
    with pytest.raises(ValueError, match="layer shapes"):
        learn.load_params(path)


def test_bf16_rounding_is_nearest_even():
    from paper_2407_20469_gb300 import learn
    f = np.array([1.0, 1.00390625, 1.01171875, -2.5, 3.0e-39, np.float32(np.inf)], dtype=np.float32)
    # 1.00390625 = 0x3F808000 is a tie -> even 0x3F80; 1.01171875 = 0x3F818000 -> 0x3F82
    assert list(learn.bf16_bits(f)) == [0x3F80, 0x3F80, 0x3F82, 0xC020, 0x0021, 0x7F80]
    v = learn.bf16_values(f)
    assert v[0] == 1.0 and v[2] == np.float32(1.015625) and v[3] == -2.5


def test_checkpoint_blob_validation():
    """apic_net_load's checks, run without a network (NULL): a well-formed BF16 blob is
    accepted; truncated, extended, mislabelled or miscounted blobs are refused."""
    from paper_2407_20469_gb300 import learn
    p = apic.pack_params(cnn.init_params(np.random.default_rng(3)))
    blob = learn.bf16_blob(p, {"epochs": 4})
    apic.validate_net_blob(blob)
    assert len(blob) == 12 + int.from_bytes(blob[8:12], "little") + 2 * p.size
    L = int.from_bytes(blob[8:12], "little")
    head = blob[12:12 + L]
    bad = {
        "truncated": blob[:-2],
        "trailing bytes": blob + b"\0\0",
        "magic": b"APICNB17" + blob[8:],
        "header length": blob[:8] + (len(blob)).to_bytes(4, "little") + blob[12:],
        "format": blob[:12] + head.replace(b"apic-net-bf16", b"apic-net-fp16") + blob[12 + L:],
        "count": blob[:12] + head.replace(str(p.size).encode(), str(p.size - 1).encode()) + blob[12 + L:],
        "short": blob[:11],
    }
    for why, b in bad.items():
        with pytest.raises(apic.ApicError) as e:
            apic.validate_net_blob(b)
        assert e.value.code == apic.APIC_EINVAL, why
