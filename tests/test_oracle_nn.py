"""Pins of the warm-start network's FP64 oracle (oracle/nn_oracle.py), on the CPU:
the convolution and the weight layout against a brute-force loop, pooling and
upsampling against their definitions, the features against explicit loops, the
gradients against finite differences (gradcheck), Adam against a hand-worked step, and
the trilinear resampling against exactly reproduced linear fields."""
import numpy as np
import pytest
import torch

from oracle import nn_oracle as nno


def test_param_count_of_the_default_network():
    # 11 convs 3x3x3 (27 cin cout + cout each) + the 1x1 head at channels 32/64/128:
    # 3488 + 27680 + 55360 + 110656 + 221312 + 2 * 442496 + 331840 + 110656 + 82976
    # + 27680 + 132 -- the ~2M-parameter network
    assert nno.param_count(32, 64, 128) == 1_856_772


def test_conv_layout_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    n, cin, cout = 4, 3, 2
    W = rng.standard_normal((cout, 27 * cin))
    b = rng.standard_normal(cout)
    X = rng.standard_normal((n, n, n, cin))  # [z][y][x][ci]
    flat_w = W.reshape(cout, 3, 3, 3, cin)
    w = torch.as_tensor(flat_w).permute(0, 4, 1, 2, 3)
    got = torch.nn.functional.conv3d(torch.as_tensor(X).permute(3, 0, 1, 2)[None], w,
                                     torch.as_tensor(b), padding=1)[0].numpy()
    for co in range(cout):
        for z in range(n):
            for y in range(n):
                for x in range(n):
                    s = b[co]
                    for kz in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                zz, yy, xx = z + kz - 1, y + ky - 1, x + kx - 1
                                if 0 <= zz < n and 0 <= yy < n and 0 <= xx < n:
                                    tap = (kz * 3 + ky) * 3 + kx
                                    s += W[co, tap * cin:(tap + 1) * cin] @ X[zz, yy, xx]
                    assert got[co, z, y, x] == pytest.approx(s, abs=1e-12)


def test_flatten_roundtrip_and_weight_permutation():
    c1, c2, c3 = 8, 8, 16
    flat = np.random.default_rng(1).standard_normal(nno.param_count(c1, c2, c3))
    layers, head = nno.unflatten(flat, c1, c2, c3)
    assert np.array_equal(nno.flatten(layers, head), flat)
    w0 = layers[0][0]  # (c1, 4, 3, 3, 3): flat index (tap * cin + ci), tap = (kz*3+ky)*3+kx
    assert w0[5, 2, 1, 0, 2].item() == flat[5 * 108 + ((1 * 3 + 0) * 3 + 2) * 4 + 2]


def test_pool_and_upsample_definitions():
    x = torch.arange(2 * 4 * 4 * 4, dtype=torch.float64).reshape(1, 2, 4, 4, 4)
    p = torch.nn.functional.avg_pool3d(x, 2)
    assert p[0, 1, 1, 0, 1].item() == x[0, 1, 2:4, 0:2, 2:4].mean().item()
    u = torch.nn.functional.interpolate(p, scale_factor=2, mode="nearest")
    assert u[0, 1, 3, 1, 2].item() == p[0, 1, 1, 0, 1].item()


def test_features():
    f = nno.features(8, [[0.3, -0.2]]).numpy()[0]
    assert f.shape == (4, 8, 8, 8)
    assert f[0, 3, 3, 0] == pytest.approx(0.5 / 8)   # x-wall node: half a cell
    assert f[0, 3, 4, 3] == pytest.approx(3.5 / 8)   # centre node
    assert (f[1, :, :, 7] == 1).all() and (f[1, :, :, 0] == -1).all() and (f[1, :, :, 1:7] == 0).all()
    assert (f[2] == 0.3).all() and (f[3] == -0.2).all()


def test_encode():
    assert np.allclose(nno.encode(10 ** 4.5, 10 ** 0.345), [0.0, 0.0])
    assert np.allclose(nno.encode(1e6, 10 ** 0.845), [1.0, 1.0])


def test_gradients_against_finite_differences():
    c1, c2, c3, n = 8, 8, 8, 8
    rng = np.random.default_rng(2)
    flat = 0.3 * rng.standard_normal(nno.param_count(c1, c2, c3))
    scal = np.array([[0.2, -0.4]])
    tgt = rng.standard_normal((1, n ** 3, 4))
    _, grads, _ = nno.loss_and_grads(flat, scal, tgt, n, c1, c2, c3)
    # central differences on a spread of parameters: h = 1e-4 keeps the O(h^2) error
    # and the rounding noise of the loss (~1e-13 / h) both below the tolerance
    idx = rng.choice(flat.size, 24, replace=False)
    h = 1e-4
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp = nno.loss_and_grads(fp, scal, tgt, n, c1, c2, c3)[0]
        lm = nno.loss_and_grads(fm, scal, tgt, n, c1, c2, c3)[0]
        assert grads[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-7), i


def test_adam_first_step_is_a_signed_learning_rate():
    # with m = v = 0 the first bias-corrected step is -lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = nno.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-2)
    assert np.allclose(p1, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_trilinear_reproduces_linear_fields_and_the_identity():
    m = 4
    c = (np.arange(m) + 0.5) / m
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = np.stack([X, 2 * Y - Z, Z, 1 + 0 * X], axis=-1).reshape(-1, 4)
    same = nno.trilinear(f, m, m, m, m).reshape(-1, 4)
    assert np.allclose(same, f, atol=1e-15)
    out = nno.trilinear(f, m, 8, 8, 8)
    cf = (np.arange(8) + 0.5) / 8
    z, y, x = np.meshgrid(cf, cf, cf, indexing="ij")
    inside = (x >= c[0]) & (x <= c[-1])
    assert np.allclose(out[..., 0][inside], x[inside], atol=1e-14)
