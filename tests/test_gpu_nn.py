"""The warm-start network's CUDA kernels (include/lbm_net.h) against the FP64 CPU oracle:
the tensor-core GEMM first.

GEMM tolerance: the operands are BF16 (exactly representable inputs on both sides) and
the products are accumulated in FP32, so |C - C_fp64| <= 2^-22 * K * sum_k |a_k b_k| per
element bounds the accumulation error with a wide margin (written below as 1e-6 * K).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def torch_mod():
    import torch
    return torch


def bf16_pair(shape_a, shape_b, seed):
    torch = torch_mod()
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(shape_a, generator=g, dtype=torch.float64).to(torch.bfloat16)
    B = torch.randn(shape_b, generator=g, dtype=torch.float64).to(torch.bfloat16)
    return A, B


def reference(A, B):
    a = A.double().numpy()
    b = B.double().numpy()
    return a @ b.T, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (256, 64, 128), (300, 100, 200),
                                   (1024, 256, 1024), (130, 16, 72), (512, 200, 640),
                                   (4096, 128, 1728),
                                   # tall 256-column GEMMs: two M tiles per CTA, ragged last pair
                                   (41000, 256, 192), (40968, 200, 136)])
def test_gemm_f32_against_fp64(M, N, K):
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    Kp = (K + 7) // 8 * 8
    A, B = bf16_pair((M, Kp), (N, Kp), M + N + K)
    A[:, K:] = 0
    B[:, K:] = 0
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32, K=K)
    ref, mag = reference(A[:, :K], B[:, :K])
    got = C.cpu().double().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= 1e-6 * K * mag + 1e-30).all()


def test_gemm_bf16_output_and_strided_operands():
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    A, B = bf16_pair((384, 256), (96, 256), 7)
    Ad, Bd = A.cuda(), B.cuda()
    # operand views with row strides 256 over K = 192, and an output with row stride 128
    C = torch.zeros((384, 128), dtype=torch.bfloat16, device="cuda")
    net.gemm_bf16(Ad[:, :192], Bd[:, :192], C[:, :96], net.GEMM_BF16, K=192)
    ref, _ = reference(A[:, :192], B[:, :192])
    got = C[:, :96].cpu().double().numpy()
    assert np.allclose(got, ref, rtol=2 ** -7, atol=1e-2)
    assert (C[:, 96:] == 0).all()


@pytest.mark.parametrize("splits", [1, 3, 8])
def test_gemm_split_k_accumulates(splits):
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    M, N, K = 256, 64, 64 * 20
    A, B = bf16_pair((M, K), (N, K), 11)
    C = torch.ones((M, N), dtype=torch.float32, device="cuda")
    net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32_ADD, splits=splits)
    ref, mag = reference(A, B)
    got = C.cpu().double().numpy() - 1.0
    assert (np.abs(got - ref) <= 1e-6 * K * mag + 1e-6).all()


def test_gemm_rejects_bad_arguments():
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    from paper_1710_04751_gb300.lbm import LBMError
    A, B = bf16_pair((128, 128), (32, 128), 3)
    C = torch.zeros((128, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(LBMError):  # split K (two K blocks) without accumulation
        net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32, splits=2)
    with pytest.raises(LBMError):  # row stride not a multiple of 8
        At = torch.zeros((128, 70), dtype=torch.bfloat16, device="cuda")
        net.gemm_bf16(At, B.cuda(), C, net.GEMM_F32, K=64)
    with pytest.raises(LBMError):  # the library's internal split-slice mode is not public
        net.gemm_bf16(A.cuda(), B.cuda(), C, 3, splits=2)


# ------------------------------------------------------------------------------------
# The network against the FP64 oracle (oracle/nn_oracle.py) on a small grid
#
# Forward: the oracle run with the CUDA path's BF16 roundings (inputs, weights, every
# stored activation) differs from the kernels only by accumulation order, so the
# relative L2 error of the output is bounded by 1e-2 (a few BF16 ulps propagated);
# without the roundings (pure FP64) by 5e-2.  Gradients: relative L2 error per layer
# 5e-2 against the rounded oracle (the kernels also round the backward GEMM operands).
# ------------------------------------------------------------------------------------

SMALL = dict(n=8, channels=(8, 16, 16))


def _small_net(seed=3, batch=2):
    from paper_1710_04751_gb300 import net
    return net.Net(n=SMALL["n"], max_batch=batch, channels=SMALL["channels"], seed=seed, lr=1e-3)


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_against_oracle():
    from oracle import nn_oracle as nno
    netw = _small_net()
    c1, c2, c3 = SMALL["channels"]
    n = SMALL["n"]
    flat = netw.get_params().astype(np.float64)
    # non-zero biases so that they are exercised
    flat_b = flat.copy()
    rng = np.random.default_rng(5)
    layers, head = nno.unflatten(flat, c1, c2, c3)
    layers = [(w, 0.05 * torch_mod().as_tensor(rng.standard_normal(b.shape[0]))) for w, b in layers]
    flat_b = nno.flatten(layers, (head[0], 0.1 * torch_mod().ones(4, dtype=torch_mod().float64)))
    netw.set_params(flat_b)
    flat_b = netw.get_params().astype(np.float64)  # the FP32 values the GPU holds
    scal = np.array([[0.3, -0.5], [-0.8, 0.6]])
    got = netw.forward(scal).cpu().double().numpy()
    layers, head = nno.unflatten(flat_b, c1, c2, c3)
    ref_q = nno.forward(layers, head, scal, n, bf16=True).numpy()
    ref = nno.forward(layers, head, scal, n, bf16=False).numpy()
    assert got.shape == (2, n ** 3, 4)
    assert _rel(got, ref_q) <= 1e-2
    assert _rel(got, ref) <= 5e-2
    netw.close()


def test_gradients_against_oracle():
    torch = torch_mod()
    from oracle import nn_oracle as nno
    netw = _small_net(seed=4)
    c1, c2, c3 = SMALL["channels"]
    n = SMALL["n"]
    rng = np.random.default_rng(6)
    scal = np.array([[0.1, 0.4], [0.7, -0.3]])
    tgt = 0.5 * rng.standard_normal((2, n ** 3, 4))
    loss = netw.gradients(scal, torch.as_tensor(tgt, dtype=torch.float32).cuda())
    g = netw.get_params(grads=True).astype(np.float64)
    flat = netw.get_params().astype(np.float64)
    tgt32 = tgt.astype(np.float32).astype(np.float64)
    ref_loss, ref_g, _ = nno.loss_and_grads(flat, scal, tgt32, n, c1, c2, c3, bf16=True)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    off = 0
    for ci, co, _ in nno.layer_shapes(c1, c2, c3):
        for size in (co * 27 * ci, co):
            assert _rel(g[off:off + size], ref_g[off:off + size]) <= 5e-2, (ci, co, size)
            off += size
    assert _rel(g[off:], ref_g[off:]) <= 5e-2  # head
    netw.close()


def test_train_step_is_one_adam_update():
    torch = torch_mod()
    from oracle import nn_oracle as nno
    netw = _small_net(seed=5)
    n = SMALL["n"]
    scal = np.array([[0.2, 0.2], [-0.5, 0.9]])
    tgt = torch.as_tensor(np.random.default_rng(7).standard_normal((2, n ** 3, 4)),
                          dtype=torch.float32).cuda()
    p0 = netw.get_params().astype(np.float64)
    netw.gradients(scal, tgt)
    g = netw.get_params(grads=True).astype(np.float64)
    netw.train_step(scal, tgt)  # same batch, same parameters: the same gradient
    p1 = netw.get_params().astype(np.float64)
    want, _, _ = nno.adam(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, lr=1e-3)
    # FP32 arithmetic; entries whose gradient is tiny may differ in sign of a rounding
    big = np.abs(g) > 1e-6
    assert np.abs(p1 - want)[big].max() <= 1e-6
    netw.close()


def test_loss_falls_when_fitting_one_sample():
    torch = torch_mod()
    netw = _small_net(seed=6, batch=1)
    n = SMALL["n"]
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    tgt = np.stack([np.sin(np.pi * x) * z, 0 * x, -np.sin(np.pi * z) * x, x - 0.5], -1)
    t = torch.as_tensor(tgt.reshape(1, -1, 4), dtype=torch.float32).cuda()
    losses = [netw.train_step([[0.1, 0.1]], t) for _ in range(300)]
    assert losses[-1] < 0.1 * losses[0]
    netw.close()


def test_training_is_bitwise_reproducible():
    # every gradient sum over voxels (split-K weight gradients, bias and head gradients, the
    # loss) is added in a fixed order, so two trainings from the same seed on the same data
    # end with identical parameters and losses
    torch = torch_mod()
    n = SMALL["n"]
    rng = np.random.default_rng(5)
    tgt = torch.as_tensor(rng.standard_normal((2, n ** 3, 4)) * 0.3, dtype=torch.float32).cuda()
    runs = []
    for _ in range(2):
        netw = _small_net(seed=4, batch=2)
        losses = [netw.train_step([[0.1, -0.2], [0.4, 0.3]], tgt) for _ in range(40)]
        runs.append((losses, netw.get_params()))
        netw.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][0][-1] < runs[0][0][0]


# ------------------------------------------------------------------------------------
# The bridge to the solver
# ------------------------------------------------------------------------------------

def _ctx(grid, seed=1, precision=None):
    import paper_1710_04751_gb300 as lbm
    return lbm.LBM(grid, 15, Ra=1e4, Pr=0.71, precision=lbm.FP64 if precision is None else precision,
                   seed=seed)


def test_set_fields_against_oracle_equilibria():
    torch = torch_mod()
    from oracle import formb
    import oracle
    sim = _ctx((5, 4, 3))
    rng = np.random.default_rng(8)
    shape = (3, 4, 5)
    rho = 1 + 0.05 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    T = rng.uniform(-0.5, 0.5, shape)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    sim.set_fields(dev(u[0]), dev(u[1]), dev(u[2]), dev(T), rho=dev(rho))
    f, g = sim.get_populations()
    cs2 = sim.params()["cs2_phi"]
    for k, j, i in [(0, 0, 0), (2, 3, 4), (1, 2, 1), (2, 0, 3)]:
        uu = u[:, k, j, i]
        assert np.abs(f[:, k, j, i] - formb.flow_equilibrium(rho[k, j, i], uu)).max() <= 1e-13
        assert np.abs(g[:, k, j, i] - formb.thermal_equilibrium(T[k, j, i], uu, 15, cs2)).max() <= 1e-13
    sim.close()


def test_targets_against_oracle_fields():
    import oracle
    sim = _ctx((8, 8, 8), seed=2)
    sim.step(40)
    from paper_1710_04751_gb300 import net
    got = net.targets(sim).cpu().double().numpy()
    F, G = sim.get_populations()
    p = oracle.Problem.cavity(8, 1e4)
    fl = p.fields(F, G)
    U0 = sim.params()["U0"]
    want = np.stack([fl["ux"] / U0, fl["uy"] / U0, fl["uz"] / U0, 2 * fl["T"]], -1).reshape(-1, 4)
    assert np.abs(got - want).max() <= 1e-6 * max(1.0, np.abs(want).max())
    sim.close()


@pytest.mark.parametrize("m,grid", [(8, (8, 8, 8)), (4, (8, 6, 5))])
def test_warm_start_sets_the_equilibria_of_the_resampled_prediction(m, grid):
    torch = torch_mod()
    from oracle import formb, nn_oracle as nno
    from paper_1710_04751_gb300 import net
    sim = _ctx(grid)
    rng = np.random.default_rng(9)
    pred = rng.uniform(-1, 1, (m ** 3, 4)).astype(np.float32)
    net.warm_start(sim, torch.as_tensor(pred).cuda(), m)
    f, g = sim.get_populations()
    U0, cs2 = sim.params()["U0"], sim.params()["cs2_phi"]
    nx, ny, nz = grid
    fields = nno.trilinear(pred.astype(np.float64), m, nx, ny, nz)
    for (k, j, i) in [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, 1, nx // 2)]:
        uu = fields[k, j, i, :3] * U0
        T = 0.5 * fields[k, j, i, 3]
        assert np.abs(f[:, k, j, i] - formb.flow_equilibrium(1.0, uu)).max() <= 1e-12
        assert np.abs(g[:, k, j, i] - formb.thermal_equilibrium(T, uu, 15, cs2)).max() <= 1e-12
    sim.close()


@pytest.mark.parametrize("iterations", [1, 4])
def test_consistent_initialisation_against_oracle(iterations):
    torch = torch_mod()
    import oracle
    from oracle import nn_oracle as nno
    grid = (6, 5, 4)
    sim = _ctx(grid)
    p = oracle.Problem.cavity(6, 1e4, ny=5, nz=4)
    rng = np.random.default_rng(10)
    shape = (4, 5, 6)
    fields = {"ux": 0.03 * rng.standard_normal(shape), "uy": 0.03 * rng.standard_normal(shape),
              "uz": 0.03 * rng.standard_normal(shape), "T": rng.uniform(-0.5, 0.5, shape)}
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    sim.set_fields(dev(fields["ux"]), dev(fields["uy"]), dev(fields["uz"]), dev(fields["T"]),
                   iterations=iterations)
    f, g = sim.get_populations()
    F, G = nno.consistent_init(p, fields, iterations)
    assert np.abs(f - F).max() <= 1e-12 and np.abs(g - G).max() <= 1e-12
    assert sim.steps_done == 0
    sim.close()


# ------------------------------------------------------------------------------------
# The implicit-GEMM convolution (lbm_nn_conv3d_bf16) against the FP64 definition: every
# output element within 1e-6 K sum |x w| (FP32 accumulation of K = 27 cin BF16 products)
# plus, for the BF16 output, its rounding (2^-8 of the value).  Grids n = 2, 4, 8 (the
# one-tile kernel: a tile spans several planes or samples) and 16, 32, 64 (the row-reuse
# kernel: 1-4 tiles of whole x-rows per CTA sharing each input box across the ky taps),
# channel counts on both operand swizzles (cin 32, 96: 64-byte rows; 64, 128, 192: 128-byte
# rows), and cout from 16 to 192 (ragged tile widths).
# ------------------------------------------------------------------------------------

CONV_CASES = [(2, 2, 32, 16), (1, 4, 64, 40), (2, 16, 32, 32), (2, 16, 96, 32),
              (2, 8, 192, 64), (1, 32, 64, 128), (3, 4, 128, 192), (1, 16, 128, 128),
              (1, 32, 192, 64), (1, 64, 96, 32), (1, 64, 32, 96)]


@pytest.mark.parametrize("B,n,cin,cout", CONV_CASES, ids=[f"b{c[0]}-n{c[1]}-ci{c[2]}-co{c[3]}" for c in CONV_CASES])
def test_implicit_convolution_against_fp64(B, n, cin, cout):
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    g = torch.Generator().manual_seed(B * 1000 + n * 10 + cin + cout)
    X = torch.randn((B, n ** 3, cin), generator=g, dtype=torch.float64).to(torch.bfloat16)
    ldw = (27 * cin + 63) // 64 * 64
    W = torch.zeros((cout, ldw), dtype=torch.float64)
    W[:, :27 * cin] = torch.randn((cout, 27 * cin), generator=g, dtype=torch.float64) / (27 * cin) ** 0.5
    W = W.to(torch.bfloat16)
    bias = (0.1 * torch.randn(cout, generator=g, dtype=torch.float64)).to(torch.float32)
    # reference: the zero-padded convolution in FP64 (weights K index tap * cin + ci)
    F = torch.nn.functional
    x = X.double().reshape(B, n, n, n, cin).permute(0, 4, 1, 2, 3)
    w = W[:, :27 * cin].double().reshape(cout, 3, 3, 3, cin).permute(0, 4, 1, 2, 3)
    y = F.conv3d(x, w, padding=1).permute(0, 2, 3, 4, 1).reshape(-1, cout)
    mag = F.conv3d(x.abs(), w.abs(), padding=1).permute(0, 2, 3, 4, 1).reshape(-1, cout)
    e = 1e-6 * 27 * cin * mag + 1e-30
    out = torch.full((B * n ** 3, cout), float("nan"), dtype=torch.float32, device="cuda")
    net.conv3d_bf16(X.cuda(), n, W.cuda(), out, mode=net.CONV_F32)
    got = out.cpu().double()
    r = ((got - y).abs() / e).max().item()
    assert r <= 1.0, r
    outb = torch.zeros((B * n ** 3, cout), dtype=torch.bfloat16, device="cuda")
    net.conv3d_bf16(X.cuda(), n, W.cuda(), outb, mode=net.CONV_BIAS_RELU_BF16, bias=bias.cuda())
    ref = torch.relu(y + bias.double())
    gotb = outb.cpu().double()
    assert ((gotb - ref).abs() <= 2.0 ** -8 * (ref.abs() + e) + e).all()


# ------------------------------------------------------------------------------------
# The implicit weight gradient (lbm_nn_conv3d_wgrad_bf16) against the FP64 definition
# dW^T[tap cin + ci][co] = sum over voxels v of X[v + shift(tap)][ci] dZ[v][co] (zero outside
# the grid): every element within (K_split + splits) 2^-24 sum |x dz| -- the first-order bound
# of FP32 summation of the split's K products and of the split partials -- after adding to
# an initial 1 (it accumulates); the padding rows 27 cin .. Kp - 1 stay at 1.  Grids from 2^3
# (one K block spans eight samples, most of them past the batch) to 128^3 (x-row segments),
# one to three samples, cin 32 / 64 / 96, cout 8 / 32 / 64 / 96 (a 128-wide tile over 96
# columns, two B boxes) / 256 (four B boxes), uneven splits.
# ------------------------------------------------------------------------------------

WGRAD_CASES = [(1, 64, 32, 32, 8), (2, 64, 96, 32, 5), (1, 64, 32, 96, 3), (1, 128, 32, 64, 16),
               (2, 32, 64, 96, 7), (3, 16, 32, 256, 2), (1, 8, 96, 8, 1), (2, 4, 32, 32, 1),
               (1, 2, 32, 64, 1)]


@pytest.mark.parametrize("B,n,cin,cout,splits", WGRAD_CASES,
                         ids=[f"b{c[0]}-n{c[1]}-ci{c[2]}-co{c[3]}-s{c[4]}" for c in WGRAD_CASES])
def test_implicit_weight_gradient_against_fp64(B, n, cin, cout, splits):
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    g = torch.Generator().manual_seed(B * 7 + n + cin * 3 + cout)
    M = B * n ** 3
    X = torch.randn((B, n ** 3, cin), generator=g, dtype=torch.float64).to(torch.bfloat16)
    dZ = (torch.randn((M, cout), generator=g, dtype=torch.float64) / 64).to(torch.bfloat16)
    Kp = (27 * cin + 63) // 64 * 64
    x = X.double().reshape(B, n, n, n, cin).numpy()
    dz = dZ.double().numpy()
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    ref = np.zeros((27 * cin, cout))
    mag = np.zeros((27 * cin, cout))
    for tap in range(27):
        kz, ky, kx = tap // 9, (tap // 3) % 3, tap % 3
        xs = xp[:, kz:kz + n, ky:ky + n, kx:kx + n, :].reshape(M, cin)
        ref[tap * cin:(tap + 1) * cin] = xs.T @ dz
        mag[tap * cin:(tap + 1) * cin] = np.abs(xs).T @ np.abs(dz)
    kblocks = -(-M // 64)
    per = -(-kblocks // splits)
    # plus the FP32 rounding of 1 + sum (the accumulation test) and of the subtraction
    bound = (per * 64 + splits) * 2.0 ** -24 * mag + 2.0 ** -23 * np.maximum(1.0, np.abs(ref)) + 1e-30
    dWT = torch.ones((Kp, cout), dtype=torch.float32, device="cuda")
    net.conv3d_wgrad_bf16(X.cuda(), n, dZ.cuda(), dWT, splits=splits)
    got = dWT.cpu().double().numpy() - 1.0
    r = np.abs(got[:27 * cin] - ref) / bound
    assert r.max() <= 1.0, (np.unravel_index(r.argmax(), r.shape), r.max())
    assert (got[27 * cin:] == 0).all()

