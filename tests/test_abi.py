"""C ABI checks that need no GPU: the library loads, exports every declared entry point,
and rejects invalid meshes on the host before touching the device."""
import os
import re

import numpy as np
import pytest

from paper_2204_04321_b300 import capi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bp_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = capi.lib()
    names = declared_entry_points()
    assert "bp_assemble_jacobian" in names and len(names) >= 8
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(capi.SIGNATURES) == names


C_TYPES = {"double": 8, "int": 4, "int32_t": 4, "int64_t": 8, "float": 4}


def header_structs():
    """{struct name: [(field, size in bytes)]} of the typedef'd structs of include/bp.h, in order."""
    src = open(os.path.join(ROOT, "include", "bp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"(?:const\s+)?(\w+)\s*(\**)\s*(.*)", decl)
            ctype, star, names = m.groups()
            for n in names.split(","):
                n = n.strip()
                ptr = star or n.startswith("*")
                n = n.lstrip("*").strip()
                count = 1
                arr = re.match(r"(\w+)\[(\d+)\]", n)
                if arr:
                    n, count = arr.group(1), int(arr.group(2))
                size = 8 if ptr else (C_TYPES[ctype] if ctype in C_TYPES else sum(z for _, z in out[ctype]))
                fields.append((n, size * count))
        out[name] = fields
    return out


@pytest.mark.parametrize("name", ["bp_params", "bp_mesh_desc", "bp_mesh_info_t", "bp_solve_opts",
                                  "bp_solve_report"])
def test_binding_structs_match_the_header(name):
    """Field names, order and sizes of the ctypes mirrors equal the C declarations."""
    import ctypes
    fields = header_structs()[name]
    cls = getattr(capi, name)
    assert [f for f, _ in cls._fields_] == [f for f, _ in fields]
    for (f, t), (_, size) in zip(cls._fields_, fields):
        assert ctypes.sizeof(t) == size, f


def test_binding_constants_match_the_header():
    src = open(os.path.join(ROOT, "include", "bp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for n, v in re.findall(r"(BP_\w+)\s*=\s*(-?\d+)", body):
            consts[n] = int(v)
    consts.update({n: int(v) for n, v in re.findall(r"#define\s+(BP_\w+)\s+(\d+)\b", src)})
    assert consts["BP_F32_ALL"] == 3 and len(consts) > 30
    for n, v in consts.items():
        if hasattr(capi, n):
            assert getattr(capi, n) == v, n
    missing = [n for n in consts if not hasattr(capi, n)]
    assert not missing, missing


def test_version_and_strerror():
    assert "sm_103a" in capi.bp_version()
    assert capi.bp_strerror(capi.BP_EMESH) == "invalid mesh"
    assert capi.bp_strerror(12345) == "unknown status"


def _upload_status(mesh):
    import ctypes
    desc, keep = capi.make_desc(mesh)
    out = ctypes.c_void_p(1)
    rc = capi.lib().bp_mesh_upload(ctypes.byref(desc), None, ctypes.byref(out))
    return rc, out.value


def tiny():
    return synth.dome_mesh(3, 2, 1, 2)


@pytest.mark.parametrize("corrupt,status", [
    (lambda m: m.tri.__setitem__((0, 1), m.nv + 5), capi.BP_EMESH),          # index out of range
    (lambda m: m.tri.__setitem__((0, slice(None)), m.tri[0, ::-1].copy()), capi.BP_EMESH),  # clockwise
    (lambda m: m.thick.__setitem__(3, 0.0), capi.BP_EMESH),                  # zero thickness
    (lambda m: m.beta.__setitem__(2, -1.0), capi.BP_EMESH),                  # negative beta
    (lambda m: m.sigma.__setitem__(1, m.sigma[2]), capi.BP_EMESH),           # sigma not increasing
    (lambda m: setattr(m.params, "n", 4.0), capi.BP_EUNSUP),                 # only n = 3
    (lambda m: m.xy.__setitem__((4, 0), np.nan), capi.BP_EMESH),             # non-finite coordinate
    (lambda m: m.tri.__setitem__((0, 2), m.tri[0, 1]), capi.BP_EMESH),        # repeated vertex
    (lambda m: m.xy.__setitem__(m.tri[0, 2], 0.5 * (m.xy[m.tri[0, 0]] + m.xy[m.tri[0, 1]])),
     capi.BP_EMESH),                                                          # collinear (zero area)
    (lambda m: setattr(m.params, "margin", 2), capi.BP_EINVAL),              # unknown margin condition
    (lambda m: (setattr(m.params, "margin", 1), setattr(m.params, "rho_w", -1.0)), capi.BP_EINVAL),
    (lambda m: setattr(m.params, "A", 0.0), capi.BP_EINVAL),                 # rate factor must be > 0
])
def test_invalid_mesh_rejected_on_host(corrupt, status):
    m = tiny()
    corrupt(m)
    rc, out = _upload_status(m)
    assert rc == status
    assert out is None


def test_null_arguments_rejected():
    import ctypes
    L = capi.lib()
    assert L.bp_mesh_upload(None, None, None) == capi.BP_EINVAL
    out = ctypes.c_void_p()
    assert L.bp_mesh_upload(None, None, ctypes.byref(out)) == capi.BP_EINVAL
    assert L.bp_mesh_info(None, None) == capi.BP_EINVAL
    assert L.bp_assemble_residual(None, None, None, None) == capi.BP_EINVAL
    assert L.bp_assemble_jacobian(None, None, None, None, 0, 0, 0, None) == capi.BP_EINVAL
    L.bp_mesh_free(None)  # no-op


def test_empty_and_oversized_meshes_rejected_before_any_device_work():
    import ctypes
    m = tiny()
    desc, keep = capi.make_desc(m)
    out = ctypes.c_void_p(1)
    desc.ntri = 0                                   # no triangles
    assert capi.lib().bp_mesh_upload(ctypes.byref(desc), None, ctypes.byref(out)) == capi.BP_EINVAL
    desc, keep = capi.make_desc(m)
    desc.nv = 1 << 30                               # 2 nv (L + 1) dofs beyond the int32 column indices
    assert capi.lib().bp_mesh_upload(ctypes.byref(desc), None, ctypes.byref(out)) == capi.BP_EINVAL
    desc, keep = capi.make_desc(m)
    desc.nlayers = 0
    assert capi.lib().bp_mesh_upload(ctypes.byref(desc), None, ctypes.byref(out)) == capi.BP_EINVAL
