"""Python binding of include/lbm_net.h (argument marshalling only): the tensor-core GEMM
building block and the learned warm-start network.  Tensors are torch CUDA tensors;
every computation runs in liblbm.so."""
import ctypes

from .lbm import LBM_OK, LBMError, load

GEMM_F32, GEMM_BF16, GEMM_F32_ADD = 0, 1, 2

# Every entry point include/lbm_net.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "lbm_nn_gemm_bf16", "lbm_net_default_config", "lbm_net_create", "lbm_net_destroy",
    "lbm_net_param_count", "lbm_net_encode", "lbm_net_get_params", "lbm_net_set_params",
    "lbm_net_forward", "lbm_net_gradients", "lbm_net_train_step", "lbm_net_last_error",
    "lbm_net_targets", "lbm_net_warm_start", "lbm_net_set_lr", "lbm_nn_gemm_timeout_probe",
    "lbm_net_tensor", "lbm_nn_conv3d_bf16", "lbm_nn_conv3d_wgrad_bf16",
)
CONV_BIAS_RELU_BF16, CONV_F32 = 0, 1

# Stored tensors (lbm_net_tensor ids): BF16 activations, then FP32 outputs and gradients.
TENSORS = ("X0", "A0", "S1", "P1", "A2", "S2", "P2", "A4", "A5", "A6", "C2", "A7", "A8", "C1",
           "A9", "A10", "OUT", "D_A10", "D_A9", "D_C1", "D_S1", "D_A8", "D_A7", "D_C2", "D_S2",
           "D_A6", "D_A5", "D_A4", "D_P2", "D_A2", "D_P1", "D_A0", "D_OUT")


class NetConfig(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("max_batch", ctypes.c_int), ("c1", ctypes.c_int),
                ("c2", ctypes.c_int), ("c3", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("cuda_stream", ctypes.c_void_p)]

_bound = False


def _lib():
    global _bound
    L = load()
    if _bound:
        return L
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    L.lbm_nn_gemm_bf16.argtypes = [vp, i64, vp, i64, vp, i64, i32, i32, i32, i32, i32, vp]
    L.lbm_net_default_config.argtypes = [P(NetConfig)]
    L.lbm_net_default_config.restype = None
    L.lbm_net_create.argtypes = [P(NetConfig), P(vp)]
    L.lbm_net_destroy.argtypes = [vp]
    L.lbm_net_destroy.restype = None
    L.lbm_net_param_count.argtypes = [vp]
    L.lbm_net_param_count.restype = i64
    L.lbm_net_encode.argtypes = [ctypes.c_double, ctypes.c_double, P(ctypes.c_float)]
    L.lbm_net_encode.restype = None
    L.lbm_net_get_params.argtypes = [vp, vp, i64, i32]
    L.lbm_net_set_params.argtypes = [vp, vp, i64]
    L.lbm_net_forward.argtypes = [vp, i32, vp, vp]
    L.lbm_net_gradients.argtypes = [vp, i32, vp, vp, P(ctypes.c_double)]
    L.lbm_net_train_step.argtypes = [vp, i32, vp, vp, P(ctypes.c_double)]
    L.lbm_net_last_error.argtypes = [vp]
    L.lbm_net_last_error.restype = ctypes.c_char_p
    L.lbm_net_targets.argtypes = [vp, vp]
    L.lbm_net_warm_start.argtypes = [vp, vp, i32, i32]
    L.lbm_net_set_lr.argtypes = [vp, ctypes.c_float]
    L.lbm_nn_gemm_timeout_probe.argtypes = [vp]
    L.lbm_net_tensor.argtypes = [vp, i32, i32, vp, i64]
    L.lbm_nn_conv3d_bf16.argtypes = [vp, i32, i32, i32, vp, i64, i32, vp, vp, i32, vp]
    L.lbm_nn_conv3d_wgrad_bf16.argtypes = [vp, i32, i32, i32, vp, i32, i32, vp, i64, i32, vp, vp]
    _bound = True
    return L


def _check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, _lib().lbm_last_error(None).decode())


def _stream(t):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def gemm_bf16(A, B, C, out_mode=GEMM_F32, splits=1, K=None):
    """C[M][N] (=, or += with GEMM_F32_ADD) A[M][K] @ B[N][K]^T; A, B bfloat16 CUDA
    tensors (row strides multiples of 8), C float32 or bfloat16."""
    M, N = C.shape
    K = A.shape[1] if K is None else K
    _check(_lib().lbm_nn_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                   C.data_ptr(), C.stride(0), M, N, K, out_mode, splits,
                                   _stream(C)))


def conv3d_bf16(X, n, W, out, mode=CONV_BIAS_RELU_BF16, bias=None):
    """3x3x3 zero-padded convolution as an implicit GEMM (lbm_nn_conv3d_bf16).  X: bfloat16
    CUDA [batch, n^3, cin] (channels last); W: bfloat16 [cout, ldw] (K = tap * cin + ci);
    out: [batch n^3, cout], bfloat16 (bias + ReLU) or float32 (CONV_F32)."""
    batch, vox, cin = X.shape
    cout = out.shape[-1]
    if vox != n ** 3:
        raise ValueError("X must hold n^3 voxels per sample")
    _check(_lib().lbm_nn_conv3d_bf16(X.data_ptr(), batch, n, cin, W.data_ptr(), W.stride(0), cout,
                                     None if bias is None else bias.data_ptr(), out.data_ptr(),
                                     int(mode), _stream(out)))


def conv3d_wgrad_bf16(X, n, dZ, dWT, splits=8):
    """dWT [Kp, cout] (float32) += the weight gradient of conv3d_bf16 as an implicit GEMM
    (lbm_nn_conv3d_wgrad_bf16), both operands read in place.  X: bfloat16 CUDA
    [batch, n^3, cin]; dZ: bfloat16 [batch n^3, cout] (the output gradient).  The split
    workspace is allocated here."""
    import torch
    batch, vox, cin = X.shape
    cout, Kp = dZ.shape[1], dWT.shape[0]
    if vox != n ** 3 or dZ.shape[0] != batch * vox or dWT.shape[1] != cout:
        raise ValueError("shapes: X [batch, n^3, cin], dZ [batch n^3, cout], dWT [Kp, cout]")
    ws = torch.empty(splits * Kp * cout, dtype=torch.float32, device=X.device)
    _check(_lib().lbm_nn_conv3d_wgrad_bf16(X.data_ptr(), batch, n, cin, dZ.data_ptr(), cout, Kp,
                                           ws.data_ptr(), ws.numel(), splits, dWT.data_ptr(), _stream(dWT)))


def gemm_timeout_probe(stream=None):
    """Run the GEMM kernel with its operand loads withheld so that its bounded wait runs
    out (lbm_nn_gemm_timeout_probe); returns the C status (LBM_ETIMEOUT when the timeout
    path works)."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    return int(_lib().lbm_nn_gemm_timeout_probe(ctypes.c_void_p(st.cuda_stream)))


def encode(Ra, Pr):
    """The network's two scalar inputs for (Ra, Pr) (lbm_net_encode)."""
    out = (ctypes.c_float * 2)()
    _lib().lbm_net_encode(float(Ra), float(Pr), out)
    return [out[0], out[1]]


def _scalars(samples):
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(samples, dtype=np.float32).reshape(-1, 2))
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def targets(sim):
    """Training targets of an LBM context's state: CUDA float32 [ncell][4] with
    (u_x, u_y, u_z) / U0 and 2 T."""
    import torch
    out = torch.empty((sim.ncell, 4), dtype=torch.float32, device=sim.device)
    sim._check(_lib().lbm_net_targets(sim._ctx, out.data_ptr()))
    return out


def warm_start(sim, pred, m, iterations=0):
    """Start an LBM context from a prediction pred (CUDA float32 [m^3][4]), with
    `iterations` rounds of the consistent initialisation."""
    import torch
    pred = pred.to(torch.float32).contiguous()
    if pred.numel() != 4 * m ** 3:
        raise ValueError("pred must hold m^3 x 4 values")
    sim._check(_lib().lbm_net_warm_start(sim._ctx, pred.data_ptr(), int(m), int(iterations)))


class Net:
    """The warm-start network on the current CUDA device (include/lbm_net.h)."""

    def __init__(self, n=64, max_batch=2, channels=(32, 64, 128), seed=1, lr=1e-3,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise LBMError(-3, "no CUDA device: the network has no CPU path")
        L = _lib()
        self._L = L
        c = NetConfig()
        L.lbm_net_default_config(ctypes.byref(c))
        c.n, c.max_batch = int(n), int(max_batch)
        c.c1, c.c2, c.c3 = (int(v) for v in channels)
        c.seed, c.lr = int(seed) & (2 ** 64 - 1), float(lr)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        c.cuda_stream = self._stream.cuda_stream
        self.n, self.max_batch, self.channels = c.n, c.max_batch, (c.c1, c.c2, c.c3)
        self._net = ctypes.c_void_p()
        rc = L.lbm_net_create(ctypes.byref(c), ctypes.byref(self._net))
        if rc != LBM_OK:
            raise LBMError(rc, L.lbm_last_error(None).decode())

    def _check(self, rc):
        if rc != LBM_OK:
            raise LBMError(rc, self._L.lbm_net_last_error(self._net).decode())

    @property
    def param_count(self):
        return int(self._L.lbm_net_param_count(self._net))

    def get_params(self, grads=False):
        import numpy as np
        out = np.empty(self.param_count, dtype=np.float32)
        self._check(self._L.lbm_net_get_params(self._net, out.ctypes.data, out.size, int(grads)))
        return out

    def set_params(self, flat):
        import numpy as np
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self._L.lbm_net_set_params(self._net, flat.ctypes.data, flat.size))

    def forward(self, scalars):
        """Predictions [B][n^3][4] (CUDA float32) for encoded scalars [B][2]."""
        import torch
        arr, ptr = _scalars(scalars)
        out = torch.empty((arr.shape[0], self.n ** 3, 4), dtype=torch.float32, device="cuda")
        self._check(self._L.lbm_net_forward(self._net, arr.shape[0], ptr, out.data_ptr()))
        return out

    def gradients(self, scalars, targets):
        arr, ptr = _scalars(scalars)
        loss = ctypes.c_double()
        t = targets.contiguous()
        self._check(self._L.lbm_net_gradients(self._net, arr.shape[0], ptr, t.data_ptr(),
                                              ctypes.byref(loss)))
        return loss.value

    def set_lr(self, lr):
        self._check(self._L.lbm_net_set_lr(self._net, float(lr)))

    def train_step(self, scalars, targets):
        arr, ptr = _scalars(scalars)
        loss = ctypes.c_double()
        t = targets.contiguous()
        self._check(self._L.lbm_net_train_step(self._net, arr.shape[0], ptr, t.data_ptr(),
                                               ctypes.byref(loss)))
        return loss.value

    def tensor(self, name, batch):
        """A stored tensor of the last call (lbm_net_tensor) as a float64 numpy array of
        shape (batch, voxels, channels); BF16 activations are widened exactly."""
        import numpy as np
        which = TENSORS.index(name)
        n, (c1, c2, c3) = self.n, self.channels
        level = {"P1": 1, "A2": 1, "S2": 1, "C2": 1, "A7": 1, "A8": 1, "D_A8": 1, "D_A7": 1,
                 "D_C2": 1, "D_S2": 1, "D_A2": 1, "D_P1": 1, "P2": 2, "A4": 2, "A5": 2, "A6": 2,
                 "D_A6": 2, "D_A5": 2, "D_A4": 2, "D_P2": 2}.get(name, 0)
        ch = {"X0": 4, "OUT": 4, "D_OUT": 4, "C2": c3 + c2, "D_C2": c3 + c2, "C1": c2 + c1,
              "D_C1": c2 + c1}
        base = name[2:] if name.startswith("D_") else name
        chans = ch.get(name) or {"A0": c1, "S1": c1, "P1": c1, "A2": c2, "S2": c2, "P2": c2,
                                 "A4": c3, "A5": c3, "A6": c3, "A7": c2, "A8": c2, "A9": c1,
                                 "A10": c1}[base]
        vox = (n >> level) ** 3
        count = batch * vox * chans
        if which <= TENSORS.index("A10"):
            raw = np.empty(count, dtype=np.uint16)
            self._check(self._L.lbm_net_tensor(self._net, which, int(batch), raw.ctypes.data, count))
            vals = (raw.astype(np.uint32) << 16).view(np.float32)  # BF16 -> FP32, exact
        else:
            vals = np.empty(count, dtype=np.float32)
            self._check(self._L.lbm_net_tensor(self._net, which, int(batch), vals.ctypes.data, count))
        return vals.astype(np.float64).reshape(batch, vox, chans)

    def close(self):
        if getattr(self, "_net", None) is not None and self._net.value:
            self._L.lbm_net_destroy(self._net)
            self._net = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
