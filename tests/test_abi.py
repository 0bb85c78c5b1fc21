"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports
every entry point include/lbm.h declares, derives the paper's parameters and rejects
invalid arguments before touching the device."""
import ctypes
import math
import os
import re

import pytest

import oracle
import paper_1710_04751_gb300 as lbm
from paper_1710_04751_gb300 import batch as batch_binding
from paper_1710_04751_gb300 import lbm as binding
from paper_1710_04751_gb300 import net as net_binding
from paper_1710_04751_gb300 import slabs as slabs_binding

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions(header):
    text = open(os.path.join(INCLUDE, header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


@pytest.mark.parametrize("header,exports", [("lbm.h", binding.EXPORTS),
                                            ("lbm_batch.h", batch_binding.EXPORTS),
                                            ("lbm_net.h", net_binding.EXPORTS),
                                            ("lbm_slabs.h", slabs_binding.EXPORTS)])
def test_library_exports_every_declared_entry_point(header, exports):
    L = binding.load()
    names = declared_functions(header)
    assert len(names) >= 1
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(exports)


def test_every_header_is_checked():
    assert sorted(f for f in os.listdir(INCLUDE) if f.endswith(".h")) == ["lbm.h", "lbm_batch.h", "lbm_net.h",
                                                                                     "lbm_slabs.h"]


def test_structure_sizes_match_header_layout():
    # lbm_params: 15+15+4+3+2 doubles then 3 ints (+4 bytes padding)
    assert ctypes.sizeof(binding.Params) == (15 + 15 + 4 + 3 + 2) * 8 + 16
    assert ctypes.sizeof(binding.Nu) == 11 * 8
    # lbm_batch_options: int (+4), u64, double, int (+4), double, 3 pointers/sizes, int,
    # the 5-int tiling, double
    assert ctypes.sizeof(batch_binding.BatchOptions) == 96
    assert ctypes.sizeof(batch_binding.Tiling) == 20
    assert ctypes.sizeof(batch_binding.Trial) == 32


@pytest.mark.parametrize("n,Ra", [(32, 1e3), (128, 1e5), (256, 1e6), (91, 1e4)])
def test_derive_params_matches_oracle(n, Ra):
    p = lbm.derive_params((n, n, n), 15, Ra, 0.71, 0.05 * math.sqrt(3.0))
    ref = oracle.physical_parameters(n, Ra, 0.71, 0.05 * math.sqrt(3.0))
    assert p.omega_f[4] == pytest.approx(ref["omega_nu"], rel=1e-14)
    assert p.omega_g[1] == pytest.approx(ref["omega_phi"], rel=1e-14)
    assert p.gbeta == pytest.approx(ref["gbeta"], rel=1e-14)
    assert p.U0 == pytest.approx(0.05, rel=1e-14)
    assert [p.omega_f[b] for b in range(4, 9)] == [p.omega_f[4]] * 5
    assert [p.omega_f[b] for b in range(9, 15)] == [1.0] * 6
    assert [p.omega_g[b] for b in range(4, 15)] == [1.0] * 11
    assert p.T_hot == 0.5 and p.T_cold == -0.5 and p.boundary == lbm.BC_CAVITY


def test_paper_parameter_values():
    # 32^3, Ra = 1e3, Pr = 0.71, U0 = 0.05
    p = lbm.derive_params((32, 32, 32), 15, 1e3, 0.71, 0.05 * math.sqrt(3.0))
    assert round(p.omega_f[4], 4) == 1.5926 and round(p.omega_g[1], 4) == 1.4703
    assert p.gbeta == pytest.approx(7.8125e-5)


@pytest.mark.parametrize("args", [
    dict(grid=(0, 4, 4)), dict(lattice=9), dict(Ra=-1.0), dict(Pr=0.0), dict(Ma=0.6),
    dict(lattice=7, cs2_phi=0.4),  # D3Q7 rest weight 1 - 3 cs2_phi < 0
])
def test_derive_params_rejects(args):
    a = dict(grid=(16, 16, 16), lattice=15, Ra=1e3, Pr=0.71, Ma=0.0866)
    a.update(args)
    with pytest.raises(lbm.LBMError) as e:
        lbm.derive_params(a["grid"], a["lattice"], a["Ra"], a["Pr"], a["Ma"],
                          **({"cs2_phi": a["cs2_phi"]} if "cs2_phi" in a else {}))
    assert e.value.code == binding.LBM_EINVAL


def test_create_rejects_bad_rates_without_touching_the_device():
    L = binding.load()
    p = lbm.derive_params((8, 8, 8), 15, 1e3, 0.71, 0.0866)
    p.omega_f[12] = 2.0
    ctx = ctypes.c_void_p()
    rc = L.lbm_create_params(ctypes.byref(binding.Grid(8, 8, 8)), 15, ctypes.byref(p), None,
                             ctypes.byref(ctx))
    assert rc == binding.LBM_EINVAL and not ctx.value
    assert b"rates" in L.lbm_last_error(None)
    p.omega_f[12] = 1.0
    p.cs2_phi = 0.4  # D3Q7 needs cs2_phi <= 1/3 (non-negative rest weight)
    rc = L.lbm_create_params(ctypes.byref(binding.Grid(8, 8, 8)), 7, ctypes.byref(p), None,
                             ctypes.byref(ctx))
    assert rc == binding.LBM_EINVAL


def test_arena_bytes():
    n = 128 ** 3
    b = lbm.arena_bytes((128, 128, 128), 15, lbm.FP32)
    # two copies of 30 populations + snapshot (4 B) + staging plane (8 B) + small scratch
    assert 2 * 30 * 4 * n + 12 * n <= b <= 2 * 30 * 4 * n + 12 * n + 64 * 1024
    assert lbm.arena_bytes((128, 128, 128), 7, lbm.FP64) > lbm.arena_bytes((128, 128, 128), 7, lbm.FP32)
    assert lbm.arena_bytes((0, 1, 1), 15, lbm.FP32) == 0


def test_noalloc_nusselt_rejects_before_touching_the_device():
    L = binding.load()
    p = lbm.derive_params((8, 8, 8), 15, 1e3, 0.71, 0.0866)
    nu = binding.Nu()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation comes first
    big = binding.Grid(4, 600, 600)  # ny * nz = 360000 > 262144 face cells of static scratch
    rc = L.lbm_nusselt_noalloc(fake, fake, 4 * 600 * 600, binding.FP32, ctypes.byref(big), 15,
                               ctypes.byref(p), None, ctypes.byref(nu))
    assert rc == binding.LBM_EINVAL
    assert b"262144" in L.lbm_last_error(None)
    small = binding.Grid(8, 8, 8)
    rc = L.lbm_nusselt_noalloc(fake, fake, 100, binding.FP32, ctypes.byref(small), 15,
                               ctypes.byref(p), None, ctypes.byref(nu))  # plane < nx*ny*nz
    assert rc == binding.LBM_EINVAL
    rc = L.lbm_nusselt_noalloc(None, fake, 512, binding.FP32, ctypes.byref(small), 15,
                               ctypes.byref(p), None, ctypes.byref(nu))
    assert rc == binding.LBM_EINVAL


def test_precision_study_error_measures():
    # the host-side measures of the precision study: relative Nusselt / peak differences
    # and max / RMS differences of the mid-plane fields (T in dT, |u| in U0)
    import numpy as np
    from paper_1710_04751_gb300 import precision
    keys = precision.NU_KEYS
    ref = {k: 2.0 for k in keys}
    got = {k: 2.02 for k in keys}
    err = precision.nu_errors(got, ref)
    assert all(abs(err[k] - 0.01) < 1e-12 for k in keys)
    a = {"T": np.zeros((4, 5)), "ux": np.zeros((4, 5)), "uy": np.zeros((4, 5)), "uz": np.zeros((4, 5))}
    b = {k: v.copy() for k, v in a.items()}
    b["T"][1, 2] = 0.3
    b["ux"][0, 0], b["uz"][0, 0] = 3.0, 4.0
    e = precision.plane_errors(a, b)
    assert e["T_max"] == 0.3 and abs(e["T_rms"] - 0.3 / np.sqrt(20)) < 1e-15
    assert e["u_max"] == 5.0 and abs(e["u_rms"] - 5.0 / np.sqrt(20)) < 1e-15


def test_checkpoint_header_layout(tmp_path):
    # lbm_checkpoint_info reads the header layout include/lbm.h documents: magic, version 1,
    # lattice, precision, grid, step count, lbm_params; anything else is rejected
    import struct
    p = binding.derive_params((12, 10, 8), 7, 1e4, 0.71, 0.05 * math.sqrt(3.0))
    head = b"LBMCKPT1" + struct.pack("<Iii3iq", 1, 7, binding.FP32, 12, 10, 8, 12345) + bytes(p)
    path = tmp_path / "c.ckpt"
    path.write_bytes(head + b"\0" * 64)
    info = binding.checkpoint_info(str(path))
    assert info["grid"] == (12, 10, 8) and info["lattice"] == 7 and info["precision"] == binding.FP32
    assert info["steps"] == 12345
    assert info["params"] == p.as_dict()
    bad = tmp_path / "bad.ckpt"
    for data in (b"LBMCKPT2" + head[8:], head[:20], b""):
        bad.write_bytes(data)
        with pytest.raises(lbm.LBMError) as e:
            binding.checkpoint_info(str(bad))
        assert e.value.code == binding.LBM_EINVAL
    with pytest.raises(lbm.LBMError):
        binding.checkpoint_info(str(tmp_path / "missing.ckpt"))


def test_slab_plan():
    # even split: the first nz % nslabs slabs take one plane more; halos at inner cuts only
    pl = slabs_binding.plan(23, 4)
    assert pl == {"z0": [0, 6, 12, 18], "nz_owned": [6, 6, 6, 5], "halo_lo": [0, 1, 1, 1],
                  "halo_hi": [1, 1, 1, 0]}
    pl = slabs_binding.plan(23, 3, owned=[1, 11, 11])
    assert pl["z0"] == [0, 1, 12] and pl["nz_owned"] == [1, 11, 11]
    # z periodic (boundary bit 2): every slab has both halos; one slab has none
    assert slabs_binding.plan(11, 4, boundary=lbm.BC_XWALLS)["halo_lo"] == [1, 1, 1, 1]
    assert slabs_binding.plan(11, 4, boundary=lbm.BC_PERIODIC)["halo_hi"] == [1, 1, 1, 1]
    assert slabs_binding.plan(11, 1, boundary=lbm.BC_PERIODIC) == {
        "z0": [0], "nz_owned": [11], "halo_lo": [0], "halo_hi": [0]}
    assert slabs_binding.plan(5, 5)["nz_owned"] == [1] * 5
    for nz, n, owned in ((5, 6, None), (5, 0, None), (0, 1, None), (6, 2, [3, 2]), (6, 2, [6, 0])):
        with pytest.raises(lbm.LBMError) as e:
            slabs_binding.plan(nz, n, owned=owned)
        assert e.value.code == binding.LBM_EINVAL


def test_slabs_create_rejects_without_touching_the_device():
    L = slabs_binding._lib()
    p = lbm.derive_params((8, 8, 8), 15, 1e3, 0.71, 0.0866)
    h = ctypes.c_void_p()
    g = binding.Grid(8, 8, 8)
    for nslabs, owned in ((0, None), (9, None), (2, [4, 5])):
        rc = L.lbm_slabs_create(ctypes.byref(g), 15, ctypes.byref(p), None, nslabs,
                                slabs_binding._ints(owned), ctypes.byref(h))
        assert rc == binding.LBM_EINVAL and not h.value
    o = binding.default_options()
    o.device_arena = 0x1000  # slabs allocate their own memory
    rc = L.lbm_slabs_create(ctypes.byref(g), 15, ctypes.byref(p), ctypes.byref(o), 2, None,
                            ctypes.byref(h))
    assert rc == binding.LBM_EINVAL and b"own device memory" in L.lbm_slabs_last_error(None)
