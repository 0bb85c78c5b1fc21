"""FP64 CPU oracle of the warm-start network and of its bridge to the solver.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU legs use
it.  It restates, in plain PyTorch CPU operations on float64 tensors (conv3d, avg-pool,
nearest upsampling, concatenation, autograd), the network that include/lbm_net.h
specifies, so that the CUDA kernels' forward pass, gradients and Adam update can be
compared with it.  The paper has no learned component: this network is an accelerator
for reaching the steady state of the method, specified by the header, not by the paper.

Layout conventions shared with the header (a data format, not arithmetic):
  * activations voxel-major, voxel = ((b*n + z)*n + y)*n + x;
  * conv weights W[cout][(tap*cin + ci)] with tap = (kz*3 + ky)*3 + kx for the input at
    (z + kz - 1, y + ky - 1, x + kx - 1);
  * flattened parameters: per layer W then b, then the head W[4][c1], b[4].

With bf16=True the forward pass rounds what the CUDA path stores in BF16 (inputs,
weights, every activation) with straight-through gradients, so that both sides take
the same rounding decisions up to accumulation order.
"""
import numpy as np
import torch
import torch.nn.functional as F

LEVELS = (0, 0, 1, 1, 2, 2, 2, 1, 1, 0, 0)


def layer_shapes(c1, c2, c3):
    cin = (4, c1, c1, c2, c2, c3, c3, c3 + c2, c2, c2 + c1, c1)
    cout = (c1, c1, c2, c2, c3, c3, c3, c2, c2, c1, c1)
    return list(zip(cin, cout, LEVELS))


def param_count(c1, c2, c3):
    return sum(co * 27 * ci + co for ci, co, _ in layer_shapes(c1, c2, c3)) + 4 * c1 + 4


def unflatten(flat, c1, c2, c3):
    """Flattened parameters -> [(w (cout, cin, 3, 3, 3), b)] per layer, head (W, b)."""
    flat = torch.as_tensor(np.asarray(flat, dtype=np.float64))
    layers, off = [], 0
    for ci, co, _ in layer_shapes(c1, c2, c3):
        W = flat[off:off + co * 27 * ci].reshape(co, 3, 3, 3, ci)
        off += co * 27 * ci
        b = flat[off:off + co]
        off += co
        layers.append((W.permute(0, 4, 1, 2, 3).contiguous(), b.clone()))
    Wh = flat[off:off + 4 * c1].reshape(4, c1)
    off += 4 * c1
    bh = flat[off:off + 4]
    return layers, (Wh.clone(), bh.clone())


def flatten(layers, head):
    parts = []
    for w, b in layers:
        co, ci = w.shape[:2]
        parts += [w.permute(0, 2, 3, 4, 1).reshape(-1), b.reshape(-1)]
    parts += [head[0].reshape(-1), head[1].reshape(-1)]
    return torch.cat(parts).detach().numpy()


def encode(Ra, Pr):
    """The two encoded scalars of a sample (header: lbm_net_encode)."""
    return np.array([(np.log10(Ra) - 4.5) / 1.5, (np.log10(Pr) - 0.345) / 0.5])


def features(n, scalars):
    """Input channels [B][4][n][n][n]: distance to the nearest half-way wall / n, the
    heated-face mask (+1 on the layer x = n-1, -1 on x = 0), the two scalars."""
    scalars = np.asarray(scalars, dtype=np.float64).reshape(-1, 2)
    i = np.arange(n) + 0.5
    d1 = np.minimum(i, n - i)
    d = np.minimum(np.minimum(d1[:, None, None], d1[None, :, None]), d1[None, None, :]) / n
    mask = np.zeros((n, n, n))
    mask[:, :, n - 1] = 1.0
    mask[:, :, 0] = -1.0
    out = np.empty((scalars.shape[0], 4, n, n, n))
    for b, (s0, s1) in enumerate(scalars):
        out[b, 0], out[b, 1], out[b, 2], out[b, 3] = d, mask, s0, s1
    return torch.as_tensor(out)


class _RoundBF16(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        return x.to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g


def _q(x, bf16):
    return _RoundBF16.apply(x) if bf16 else x


def forward(layers, head, scalars, n, bf16=False):
    """Outputs [B][n^3][4] (voxel-major) of the network for the encoded scalars."""
    x = _q(features(n, scalars), bf16)

    def conv(x, l):
        w, b = layers[l]
        return _q(F.relu(F.conv3d(x, _q(w, bf16), b, padding=1)), bf16)

    a0 = conv(x, 0)
    s1 = conv(a0, 1)
    p1 = _q(F.avg_pool3d(s1, 2), bf16)
    a2 = conv(p1, 2)
    s2 = conv(a2, 3)
    p2 = _q(F.avg_pool3d(s2, 2), bf16)
    a4 = conv(p2, 4)
    a5 = conv(a4, 5)
    a6 = conv(a5, 6)
    c2 = torch.cat([F.interpolate(a6, scale_factor=2, mode="nearest"), s2], dim=1)
    a7 = conv(c2, 7)
    a8 = conv(a7, 8)
    c1 = torch.cat([F.interpolate(a8, scale_factor=2, mode="nearest"), s1], dim=1)
    a9 = conv(c1, 9)
    a10 = conv(a9, 10)
    Wh, bh = head
    out = torch.einsum("oc,bczyx->bzyxo", Wh, a10) + bh
    return out.reshape(out.shape[0], -1, 4)


def loss_and_grads(flat, scalars, targets, n, c1, c2, c3, bf16=False):
    """Mean squared error against targets [B][n^3][4] and its gradient, flattened."""
    layers, head = unflatten(flat, c1, c2, c3)
    params = [t for wb in layers for t in wb] + list(head)
    for t in params:
        t.requires_grad_(True)
    out = forward(layers, head, scalars, n, bf16)
    tgt = torch.as_tensor(np.asarray(targets, dtype=np.float64)).reshape(out.shape)
    loss = ((out - tgt) ** 2).mean()
    loss.backward()
    grads = flatten([(w.grad, b.grad) for w, b in layers], (head[0].grad, head[1].grad))
    return float(loss.detach()), grads, out.detach().numpy()


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) in float64."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def trilinear(pred, m, nx, ny, nz):
    """A cell-centred m^3 field [m^3][4] sampled at the nodes of an nx x ny x nz grid
    (node i at (i + 1/2)/nx of the box; outside the outermost cell centres the edge
    value), by the textbook trilinear formula, one node at a time."""
    P = np.asarray(pred, dtype=np.float64).reshape(m, m, m, 4)
    out = np.empty((nz, ny, nx, 4))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                s = [(i + 0.5) * m / nx - 0.5, (j + 0.5) * m / ny - 0.5, (k + 0.5) * m / nz - 0.5]
                lo, w = [], []
                for v in s:
                    v = min(max(v, 0.0), m - 1.0)
                    l0 = min(int(np.floor(v)), max(m - 2, 0))
                    lo.append(l0)
                    w.append(0.0 if m == 1 else v - l0)
                acc = np.zeros(4)
                for dz in (0, 1):
                    for dy in (0, 1):
                        for dx in (0, 1):
                            wt = ((w[0] if dx else 1 - w[0]) * (w[1] if dy else 1 - w[1])
                                  * (w[2] if dz else 1 - w[2]))
                            if wt:
                                acc += wt * P[lo[2] + dz, lo[1] + dy, lo[0] + dx]
                out[k, j, i] = acc
    return out


def consistent_init(problem, fields, iterations, rho=None):
    """The consistent initialisation the solver header specifies, in the oracle: the
    populations of the equilibria of `fields` (ux, uy, uz, T arrays [nz][ny][nx]), then
    `iterations` (rounded up to even) rounds of one oracle step and
    p <- p - p_eq(current u, T) + p_eq(given u, T) at every node, rho kept.  Equilibria
    from oracle/formb.py; u and T of a stored state as the oracle's fields() defines them."""
    from oracle import formb
    nx, ny, nz = problem.nx, problem.ny, problem.nz
    q = problem.q_g
    cs2 = problem.cs2_phi
    ux, uy, uz, T = (np.asarray(fields[k], dtype=np.float64) for k in ("ux", "uy", "uz", "T"))
    F = np.empty((15, nz, ny, nx))
    G = np.empty((q, nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                u = (ux[k, j, i], uy[k, j, i], uz[k, j, i])
                r = 1.0 if rho is None else rho[k, j, i]
                F[:, k, j, i] = formb.flow_equilibrium(r, u)
                G[:, k, j, i] = formb.thermal_equilibrium(T[k, j, i], u, q, cs2)
    for _ in range(iterations + (iterations & 1)):
        F, G = problem.step(F, G)
        cur = problem.fields(F, G)
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    r = cur["rho"][k, j, i]
                    uc = (cur["ux"][k, j, i], cur["uy"][k, j, i], cur["uz"][k, j, i])
                    ut = (ux[k, j, i], uy[k, j, i], uz[k, j, i])
                    F[:, k, j, i] += formb.flow_equilibrium(r, ut) - formb.flow_equilibrium(r, uc)
                    G[:, k, j, i] += (formb.thermal_equilibrium(T[k, j, i], ut, q, cs2)
                                      - formb.thermal_equilibrium(cur["T"][k, j, i], uc, q, cs2))
    return F, G
