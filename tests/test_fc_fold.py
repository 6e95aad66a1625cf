"""Host-side check of the polynomial network's folding: a network with the
learned quadratic activation z + alpha z^2 and the pure-square network that
mmfhe_fold_poly_net makes of it (the form the encrypted FC circuit runs)
compute the same outputs."""
import numpy as np
import pytest

from oracle import circuits as cc


def quad_forward(w, dims, alpha, x):
    v, off = np.asarray(x, dtype=np.float64), 0
    for l in range(len(dims) - 1):
        a, b = dims[l], dims[l + 1]
        W = w[off: off + b * (a + 1)].reshape(b, a + 1).astype(np.float64)
        off += b * (a + 1)
        z = W[:, :a] @ v + W[:, a]
        v = z + alpha * z * z if l < len(dims) - 2 else z
    return v


@pytest.mark.parametrize("dims", [(120, 32, 16, 6), (10, 4), (7, 5, 3)])
def test_fold_equals_quadratic_network(dims):
    import paper_2603_22437_b300 as M
    g = np.random.default_rng(sum(dims))
    alpha = float(np.float32(0.1))   # the ABI takes alpha as a float
    nw = sum(dims[l + 1] * (dims[l] + 1) for l in range(len(dims) - 1))
    w = g.normal(0, 0.3, nw).astype(np.float32)
    mats = M.fold_poly_net(dims, alpha, w, 128)
    for l in range(len(dims) - 1):
        assert mats[l][127, 127] == 1.0 and not mats[l][127, :127].any()
    for s in range(5):
        x = g.normal(size=dims[0])
        ref = quad_forward(w, dims, alpha, x)
        got = cc.fc_forward(mats, x, 128)[: dims[-1]]
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_fold_rejects_bad_shapes():
    import paper_2603_22437_b300 as M
    w = np.zeros(200 * 129, dtype=np.float32)
    with pytest.raises(M.MmfheError):
        M.fold_poly_net((128, 6), 0.1, w, 128)   # a width not below D
    with pytest.raises(M.MmfheError):
        M.fold_poly_net((10, 4), 0.1, w, 100)    # D not a power of two


def test_fold_wide_first_layer_equals_quadratic_network():
    """A gesture plan's FC1 reads more inputs than the slot period: the wide
    fold composed with the gesture chain's FP64 network equals the
    quadratic-activation network."""
    import paper_2603_22437_b300 as M
    cfg = cc.GestureConfig(antennas=2, bins=4, chirps=8, fc_dims=(7, 5, 3), width=16)
    dims = (cfg.ard,) + tuple(cfg.fc_dims)
    g = np.random.default_rng(8)
    alpha = float(np.float32(0.25))
    nw = sum(dims[l + 1] * (dims[l] + 1) for l in range(len(dims) - 1))
    w = g.normal(0, 0.2, nw).astype(np.float32)
    first, tail = M.fold_poly_net_wide(dims, alpha, w, cfg.width)
    assert first.shape == (16, cfg.ard + 1) and tail.shape == (2, 16, 16)
    assert first[15, cfg.ard] == 1.0 and not first[15, : cfg.ard].any()
    for s in range(4):
        feat = g.normal(size=(cfg.antennas, cfg.bins, cfg.chirps))
        ref = quad_forward(w, dims, alpha, feat.reshape(-1))
        got = cc.gesture_forward([first, tail[0], tail[1]], feat, cfg)[: dims[-1]]
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    with pytest.raises(M.MmfheError):
        M.fold_poly_net_wide((64, 16, 6), 0.1, w, 16)   # a hidden width not below D
