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
