"""The warm-start network at its production channel widths (32, 64, 128) on a 16^3 and a
24^3 grid, batch 2, checked element by element: every stored activation, the outputs,
every activation gradient and every parameter gradient.

Each layer is recomputed in FP64 (torch CPU, the definitions the oracle uses: zero-padded
3x3x3 convolution, bias, ReLU, 2x average pooling, nearest upsampling, concatenation,
the 1x1 head, the mean squared error) from the GPU's OWN stored inputs of that layer
(lbm_net_tensor), so that a difference in one layer cannot hide behind, or spread into,
another.  At 16^3 every convolution takes the implicit kernels of the 64^3 training (tile
widths BN = 32 ... 128, the row-reuse form, split-K weight gradients); 24^3 is not a power
of two, so there every convolution takes the explicit im2col matrix and the GEMM, the
fallback, with the first layer's input in its padded 32-channel rows.

Per-element bounds, from the arithmetic: a product sum of K BF16 x BF16 terms accumulated
in FP32 on the tensor cores differs from the FP64 sum by at most 1e-6 K sum |a b| (as in
the GEMM tests); a value stored in BF16 adds its rounding, 2^-8 of its size; FP32 sums
of K terms add at most 1e-6 K sum |terms|.  ReLU is 1-Lipschitz.  The ReLU masks and the
BF16 rounding of the backward GEMM operand dZ = bf16(dA [A > 0]) are recomputed from the
GPU's own FP32 dA and BF16 A, so both sides take the same decisions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRIDS, BATCH, CH = (16, 24), 2, (32, 64, 128)
U8 = 2.0 ** -8   # relative rounding of a BF16 store (8 significant bits, round to nearest)
U24 = 2.0 ** -24


def _torch():
    import torch
    return torch


def _q(t):
    torch = _torch()
    return t.to(torch.bfloat16).to(torch.float64)  # round to nearest even, as the kernels


def _grid(a, m):
    """(B, voxels, C) -> (B, C, z, y, x)"""
    torch = _torch()
    return torch.as_tensor(a).reshape(BATCH, m, m, m, -1).permute(0, 4, 1, 2, 3).contiguous()


def _assert_within(got, ref, bound, what):
    got, ref, bound = (np.asarray(x, dtype=np.float64) for x in (got, ref, bound))
    r = np.abs(got - ref) / (bound + 1e-30)
    i = np.unravel_index(r.argmax(), r.shape)
    assert r.max() <= 1.0, f"{what}: worst {r.max():.3g} x bound at {i} (got {got[i]!r}, ref {ref[i]!r})"
    return r.max()


@pytest.fixture(scope="module", params=GRIDS, ids=[f"n{g}" for g in GRIDS])
def run(request):
    N_GRID = request.param
    torch = _torch()
    from oracle import nn_oracle as nno
    from paper_1710_04751_gb300 import net
    netw = net.Net(n=N_GRID, max_batch=BATCH, channels=CH, seed=7, lr=1e-3)
    c1, c2, c3 = CH
    # non-zero biases, so that the bias paths are exercised
    flat = netw.get_params().astype(np.float64)
    layers, head = nno.unflatten(flat, c1, c2, c3)
    rng = np.random.default_rng(11)
    layers = [(w, torch.as_tensor(0.05 * rng.standard_normal(b.shape[0]))) for w, b in layers]
    netw.set_params(nno.flatten(layers, (head[0], torch.as_tensor(0.1 * rng.standard_normal(4)))))
    scal = np.array([[0.3, -0.5], [-0.8, 0.6]], dtype=np.float32)
    tgt = (0.5 * rng.standard_normal((BATCH, N_GRID ** 3, 4))).astype(np.float32)
    loss = netw.gradients(scal, torch.as_tensor(tgt).cuda())
    t = {name: netw.tensor(name, BATCH) for name in net.TENSORS}
    params = netw.get_params().astype(np.float64)
    grads = netw.get_params(grads=True).astype(np.float64)
    netw.close()
    layers, head = nno.unflatten(params, c1, c2, c3)
    glayers, ghead = nno.unflatten(grads, c1, c2, c3)
    return dict(t=t, layers=layers, head=head, glayers=glayers, ghead=ghead, scal=scal, tgt=tgt,
                loss=loss, n=N_GRID)


# layer l: (input tensor, output tensor, grid level)
CONVS = [("X0", "A0", 0), ("A0", "S1", 0), ("P1", "A2", 1), ("A2", "S2", 1), ("P2", "A4", 2),
         ("A4", "A5", 2), ("A5", "A6", 2), ("C2", "A7", 1), ("A7", "A8", 1), ("C1", "A9", 0),
         ("A9", "A10", 0)]
# layer l backward: where the GPU wrote the gradient of its input (None for layer 0)
DX = ["", "D_A0", "D_P1", "D_A2", "D_P2", "D_A4", "D_A5", "D_C2", "D_A7", "D_C1", "D_A9"]


def test_input_features_exact(run):
    torch = _torch()
    from oracle import nn_oracle as nno
    ref = _q(nno.features(run["n"], run["scal"].astype(np.float64)))
    got = _grid(run["t"]["X0"], run["n"])
    assert torch.equal(got, ref)


@pytest.mark.parametrize("l", range(11))
def test_convolution_outputs(run, l):
    torch = _torch()
    F = torch.nn.functional
    src, dst, level = CONVS[l]
    m = run["n"] >> level
    X = _grid(run["t"][src], m)
    A = _grid(run["t"][dst], m)
    w, b = run["layers"][l]
    wq = _q(w)
    y = F.conv3d(X, wq, b, padding=1)
    mag = F.conv3d(X.abs(), wq.abs(), b.abs(), padding=1)
    K = 27 * X.shape[1]
    eacc = 1e-6 * K * mag + U24 * mag
    r = torch.relu(y)
    _assert_within(A, r, U8 * (r + eacc) + eacc, f"layer {l} output")
    assert (A >= 0).all()


@pytest.mark.parametrize("src,dst,level", [("S1", "P1", 0), ("S2", "P2", 1)])
def test_pooling(run, src, dst, level):
    torch = _torch()
    F = torch.nn.functional
    m = run["n"] >> level
    S = _grid(run["t"][src], m)
    P = _grid(run["t"][dst], m // 2)
    ref = F.avg_pool3d(S, 2)
    e = 8 * U24 * F.avg_pool3d(S.abs(), 2)
    _assert_within(P, ref, U8 * (ref.abs() + e) + e, dst)


def test_concatenations_exact(run):
    torch = _torch()
    F = torch.nn.functional
    t = run["t"]
    c1, c2, c3 = CH
    up = lambda a: F.interpolate(a, scale_factor=2, mode="nearest")  # noqa: E731
    C2 = _grid(t["C2"], run["n"] // 2)
    assert torch.equal(C2[:, :c3], up(_grid(t["A6"], run["n"] // 4)))
    assert torch.equal(C2[:, c3:], _grid(t["S2"], run["n"] // 2))
    C1 = _grid(t["C1"], run["n"])
    assert torch.equal(C1[:, :c2], up(_grid(t["A8"], run["n"] // 2)))
    assert torch.equal(C1[:, c2:], _grid(t["S1"], run["n"]))


def test_head_loss_and_their_gradients(run):
    t = run["t"]
    Wh, bh = (x.numpy() for x in run["head"])
    A10 = t["A10"].reshape(-1, CH[0])
    out = t["OUT"].reshape(-1, 4)
    ref = A10 @ Wh.T + bh
    mag = np.abs(A10) @ np.abs(Wh).T + np.abs(bh)
    _assert_within(out, ref, 1e-6 * (CH[0] + 1) * mag, "head output")
    tgt = run["tgt"].reshape(-1, 4).astype(np.float64)
    count = out.size
    d = out - tgt
    assert run["loss"] == pytest.approx(np.mean(d * d), rel=1e-6)
    dOut = t["D_OUT"].reshape(-1, 4)
    _assert_within(dOut, 2.0 * d / count, 4 * U24 * np.abs(2.0 * d / count) + 1e-30, "dOut")
    # gradients of the head from the GPU's dOut: dA10, then the head's parameters
    dA10 = t["D_A10"].reshape(-1, CH[0])
    _assert_within(dA10, dOut @ Wh, 1e-6 * 4 * (np.abs(dOut) @ np.abs(Wh)), "dA10")
    M = dOut.shape[0]
    gWh, gbh = (x.numpy() for x in run["ghead"])
    _assert_within(gWh, dOut.T @ A10, 1e-6 * M * (np.abs(dOut).T @ np.abs(A10)), "head dW")
    _assert_within(gbh, dOut.sum(axis=0), 1e-6 * M * np.abs(dOut).sum(axis=0), "head db")


@pytest.mark.parametrize("l", range(11))
def test_convolution_gradients(run, l):
    torch = _torch()
    tg = torch.nn.grad
    t = run["t"]
    src, dst, level = CONVS[l]
    m = run["n"] >> level
    X = _grid(t[src], m)
    A = _grid(t[dst], m)
    dA = _grid(t["D_" + dst], m)
    w, _ = run["layers"][l]
    wq = _q(w)
    g = dA * (A > 0)                       # FP32 values, exact in FP64
    dZ = _q(g.to(torch.float32).to(torch.float64))  # the BF16 GEMM operand
    M = BATCH * m ** 3
    # bias gradient: FP32 sums of g over the voxels
    gw, gb = run["glayers"][l]
    _assert_within(gb, g.sum(dim=(0, 2, 3, 4)), 1e-6 * M * g.abs().sum(dim=(0, 2, 3, 4)), f"layer {l} db")
    # weight gradient: sum over voxels of X (x) dZ, split K over voxels
    ref = tg.conv3d_weight(X, w.shape, dZ, padding=1)
    mag = tg.conv3d_weight(X.abs(), w.shape, dZ.abs(), padding=1)
    _assert_within(gw, ref, 1e-6 * M * mag + 1e-30, f"layer {l} dW")
    if l > 0:  # input gradient: the convolution of dZ with the mirrored weights
        dX = _grid(t[DX[l]], m)
        ref = tg.conv3d_input(X.shape, wq, dZ, padding=1)
        mag = tg.conv3d_input(X.shape, wq.abs(), dZ.abs(), padding=1)
        K = 27 * A.shape[1]
        _assert_within(dX, ref, 1e-6 * K * mag + 1e-30, f"layer {l} dX")


@pytest.mark.parametrize("cat,up_from,skip,split,level", [
    ("D_C1", "D_A8", "D_S1", CH[1], 0), ("D_C2", "D_A6", "D_S2", CH[2], 1)])
def test_upsampling_and_skip_gradients(run, cat, up_from, skip, split, level):
    torch = _torch()
    F = torch.nn.functional
    t = run["t"]
    m = run["n"] >> level
    dC = _grid(t[cat], m)
    # nearest upsampling: the coarse gradient sums its 8 fine children (FP32)
    ref = 8 * F.avg_pool3d(dC[:, :split], 2)
    mag = 8 * F.avg_pool3d(dC[:, :split].abs(), 2)
    _assert_within(_grid(t[up_from], m // 2), ref, 8 * U24 * mag + 1e-30, up_from)
    # skip connection: its slice of the concatenation plus the pooling's share
    dP = _grid(t["D_P1" if level == 0 else "D_P2"], m // 2)
    share = 0.125 * F.interpolate(dP, scale_factor=2, mode="nearest")
    ref = dC[:, split:] + share
    _assert_within(_grid(t[skip], m), ref, 2 * U24 * (dC[:, split:].abs() + share.abs()) + 1e-30, skip)
