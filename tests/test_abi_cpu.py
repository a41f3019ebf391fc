"""Host-side checks of the C ABI (no GPU): the library loads, exports every function that
include/strm.h declares, and the binding's ctypes structs match the header's layout."""
import ctypes
import os
import re

import pytest

from paper_2004_02276_gb300 import binding, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "strm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(strm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.SIGNATURES)


def test_struct_field_counts_match_header():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for cname, py in (("strm_grid", binding.Grid), ("strm_phys", binding.Phys),
                      ("strm_scheme", binding.Scheme)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + cname + ";", text).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            typ, names = decl.split(None, 1)
            fields += [(typ, n.strip()) for n in names.split(",")]
        assert [n for _, n in fields] == [f for f, _ in py._fields_], cname
        for (typ, _), (_, ct) in zip(fields, py._fields_):
            assert {"int": ctypes.c_int, "double": ctypes.c_double}[typ] == ct


def test_workspace_bytes_rejects_invalid(lib):
    g, p, s = binding.structs(inputs.C1)
    ok = lib.strm_workspace_bytes(ctypes.byref(g), ctypes.byref(s))
    assert ok > 0
    for bad in (inputs.C1.replace(nx=0), inputs.C1.replace(L=4), inputs.C1.replace(lx=-1.0)):
        gb, _, sb = binding.structs(bad)
        assert lib.strm_workspace_bytes(ctypes.byref(gb), ctypes.byref(sb)) == 0
    # the workspace grows with the grid
    g2, _, s2 = binding.structs(inputs.C2)
    assert lib.strm_workspace_bytes(ctypes.byref(g2), ctypes.byref(s2)) > 10 * ok


def test_init_rejects_bad_arguments_before_any_cuda_call(lib):
    g, p, s = binding.structs(inputs.C1)
    ctx = ctypes.c_void_p()
    # null workspace
    rc = lib.strm_init_grid(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), ctypes.byref(s),
                            None, 0, None)
    assert rc == -1 and b"workspace" in lib.strm_last_error()
    # misaligned workspace pointer (never dereferenced: rejected on the host)
    rc = lib.strm_init_grid(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), ctypes.byref(s),
                            ctypes.c_void_p(0x1008), 1 << 40, None)
    assert rc == -1 and b"aligned" in lib.strm_last_error()
    # too small
    rc = lib.strm_init_grid(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), ctypes.byref(s),
                            ctypes.c_void_p(0x1000), 16, None)
    assert rc == -4
    # bad physics
    p.gamma = 1.0
    rc = lib.strm_init_grid(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), ctypes.byref(s),
                            ctypes.c_void_p(0x1000), 1 << 40, None)
    assert rc == -1
    assert lib.strm_set_bc(None, 0, 1, None, 0) == -1
    lib.strm_destroy(None)


def test_host_side_argument_checks(lib):
    """Calls that fail before touching a device: null pointers and bad sizes or bits return
    STRM_EINVAL with a message, and the binding refuses host tensors for the conversions."""
    import torch

    assert lib.strm_convert_f64_f32(None, None, -1, None) == -1
    assert lib.strm_convert_f32_f64(None, None, 5, None) == -1
    assert lib.strm_convert_f64_f32(None, None, 0, None) == 0  # nothing to do
    assert lib.strm_set_overlap(None, 1) == -1
    assert b"conversion" in lib.strm_last_error() or b"context" in lib.strm_last_error()
    with pytest.raises(ValueError):
        binding.convert(torch.zeros(4, dtype=torch.float64))


def test_face_settings_of_the_workloads():
    """The (face, kind, params) calls the binding makes for each boundary configuration."""
    F, K = binding.FACES, binding.BC_KINDS
    ch = binding.face_settings(inputs.C1)
    assert ch == [(F["xmin"], K["periodic"], None), (F["xmax"], K["periodic"], None),
                  (F["ymin"], K["wall"], None), (F["ymax"], K["wall"], None)]
    c4 = inputs.C4
    got = {face: (kind, params) for face, kind, params in binding.face_settings(c4)}
    ref = [1.0, 1.0, 0.0, 0.0, c4.r_gas]
    assert got[F["xmin"]] == (K["recycle"], ref + [float(c4.i_recycle), c4.delta_in])
    assert got[F["xmax"]] == (K["char"], ref)
    assert got[F["ymin"]] == (K["wall"], None)
    assert got[F["ymax"]] == (K["shock"], ref + [c4.shock_theta, c4.shock_ximp])
    # the digital-filter inflow face is set with its profiles, not by strm_set_bc
    df = inputs.PAPER_BL
    assert F["xmin"] not in [f for f, _, _ in binding.face_settings(df)]
    g, p, s = binding.structs(df)
    assert (g.y_map, s.L, p.visc_law) == (binding.Y_MAPS["sinh1"], 2, binding.VISC_LAWS["sutherland"])
    with pytest.raises(ValueError):
        binding.face_settings(inputs.C1.replace(bc_xmin="bogus"))


def test_static_totals_binding_rejects_bad_state_before_the_library():
    """The binding of the allocation-free totals checks the state (contiguous float64 CUDA
    tensor of shape [5, nz, ny, nx]) before any call into the library, so that a mis-sized,
    FP32 or host tensor never reaches a kernel."""
    import torch

    case = inputs.Case(nx=8, ny=6, nz=4)
    for bad in (torch.zeros(8, dtype=torch.float64),
                torch.zeros((5, 4, 6, 8), dtype=torch.float64),       # host memory
                torch.zeros((5, 4, 6, 8), dtype=torch.float32)):
        with pytest.raises(ValueError):
            binding.conserved_totals_static(case, bad)
