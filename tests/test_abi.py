"""CPU checks of the C ABI: the library builds and loads, exports every function the
header declares, and the host-side type setup validates meshes and materials."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2011_04332_b300 import build, inputs as I, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native.load_library()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*npfem_status\s+(npfem_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("npfem_create_cell_type", "npfem_destroy_cell_type", "npfem_batch_create",
                     "npfem_step", "npfem_step_host", "npfem_last_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    cdll = ctypes.CDLL(native.LIB_PATH)
    for name in declared_functions():
        assert hasattr(cdll, name), f"{name} declared in include/ but not exported"


def test_analyze_reports_factor_statistics(lib):
    m = I.rbc_mesh(3)
    info = native.analyze_cell_type(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), I.DT_DEFAULT)
    assert info["n_verts"] == 642 and info["n_tris"] == 1280 and info["n_hinges"] == 1920
    # a fill-reducing ordering keeps the factor far below the dense n(n-1)/2
    assert 0 < info["nnz_factor"] < 0.2 * 642 * 641 / 2
    assert info["total_mass"] == pytest.approx(1.1 * info["rest_volume"], rel=1e-12)


def _max_elements_at_a_vertex(n, elems):
    return int(np.bincount(np.asarray(elems).ravel(), minlength=n).max())


def test_element_colour_classes(lib):
    """Triangles and hinges come in vertex-disjoint colour classes (verified as built);
    a valid class count is at least the largest number of elements at one vertex, and the
    DSatur colouring stays within a few classes of that bound on the workload meshes (it
    finds 9-10 triangle classes against a bound of 6, 16-17 hinge classes against 10-12).
    A mesh that would need more than 64 classes reports 0 (its type runs the one-warp
    iteration kernels)."""
    from oracle import npfem_oracle as O
    for m in (I.platelet_mesh(2), I.rbc_mesh(2), I.rbc_mesh(3), I.rbc_mesh(4)):
        info = native.analyze_cell_type(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), I.DT_DEFAULT)
        n = m.verts.shape[0]
        hinges = O.rest_state(m.verts, m.tris, *I.RBC_MATERIAL.as_tuple(), I.DT_DEFAULT).hinges
        lo_t, lo_h = _max_elements_at_a_vertex(n, m.tris), _max_elements_at_a_vertex(n, hinges)
        assert lo_t <= info["tri_colours"] <= lo_t + 5, (m.name, info["tri_colours"], lo_t)
        assert lo_h <= info["hinge_colours"] <= lo_h + 7, (m.name, info["hinge_colours"], lo_h)
    m = I.bipyramid(70)
    info = native.analyze_cell_type(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), I.DT_DEFAULT)
    assert info["tri_colours"] == 0 and info["hinge_colours"] == 0
    assert info["n_tris"] == 140


def test_ordering_fill_on_the_workload_meshes(lib):
    """The fill-reducing ordering (least fill among plane-cut nested dissections with
    one-sided and cut-cover separators, the latter reordered by constrained minimum
    degree, and exact minimum degree up to 1500 vertices) keeps nnz(L) of the workload
    meshes at the values it reaches: the FP64 solve's work is 12 nnz(L) + 3n per
    cell-solve, so a regression here is a slower step."""
    for m, bound in ((I.platelet_mesh(2), 4226), (I.rbc_mesh(3), 27615), (I.rbc_mesh(4), 161174)):
        info = native.analyze_cell_type(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), I.DT_DEFAULT)
        assert info["nnz_factor"] <= bound, (m.name, info["nnz_factor"], bound)


def test_analyze_matches_oracle_rest_quantities(lib):
    from oracle import npfem_oracle as O
    for m in (I.tetrahedron(), I.icosahedron(), I.platelet_mesh(1), I.rbc_mesh(2)):
        info = native.analyze_cell_type(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), 0.1)
        rs = O.rest_state(m.verts, m.tris, *I.RBC_MATERIAL.as_tuple(), 0.1)
        assert info["rest_area"] == pytest.approx(rs.A0, rel=1e-13)
        assert info["rest_volume"] == pytest.approx(rs.V0, rel=1e-13)
        assert info["n_hinges"] == rs.hinges.shape[0]


def _expect(code, fn):
    with pytest.raises(native.NpfemError) as ei:
        fn()
    assert ei.value.code == code, str(ei.value)


def test_bad_meshes_are_rejected(lib):
    m = I.icosahedron()
    mat = I.RBC_MATERIAL.as_tuple()
    # open mesh: drop a triangle
    _expect(-2, lambda: native.analyze_cell_type(m.verts, m.tris[:-1], mat, 0.1))
    # inconsistent orientation: flip one triangle
    t = m.tris.copy()
    t[0] = t[0][[0, 2, 1]]
    _expect(-2, lambda: native.analyze_cell_type(m.verts, t, mat, 0.1))
    # index out of range
    t = m.tris.copy()
    t[3, 1] = 99
    _expect(-2, lambda: native.analyze_cell_type(m.verts, t, mat, 0.1))
    # degenerate rest triangle (two coincident vertices)
    v = m.verts.copy()
    v[m.tris[0, 1]] = v[m.tris[0, 0]]
    _expect(-2, lambda: native.analyze_cell_type(v, m.tris, mat, 0.1))
    # inward orientation: negative volume
    _expect(-2, lambda: native.analyze_cell_type(m.verts, m.tris[:, [0, 2, 1]], mat, 0.1))


def test_invalid_arguments_are_rejected(lib):
    m = I.icosahedron()
    _expect(-1, lambda: native.analyze_cell_type(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), -1.0))
    _expect(-1, lambda: native.analyze_cell_type(m.verts, m.tris, (1, .05, 10, 10, 0.0), 0.1))


def test_binding_status_bits_match_the_header():
    """The binding's NPFEM_CELL_* values are the header's."""
    hdr = open(os.path.join(ROOT, "include", "npfem.h")).read()
    bits = {k: int(v) for k, v in re.findall(r"#define NPFEM_CELL_(\w+) (\d+)", hdr)}
    assert len(bits) == 6
    for k, v in bits.items():
        if k != "OK":
            assert getattr(native, "CELL_" + k) == v, k


def test_vertex_limit_is_enforced(lib):
    """Types are limited to 65535 vertices (the packed solve tables hold 16-bit row
    indices): one more is refused as unsupported before any mesh work."""
    m = I.icosahedron()
    v = np.zeros((65536, 3))
    v[:12] = m.verts
    _expect(-6, lambda: native.analyze_cell_type(v, m.tris, I.RBC_MATERIAL.as_tuple(), 0.1))


def test_strain_limits_are_checked_on_the_host(lib):
    """Both 0 (or both 1) select the rotations; otherwise 0 < s_min <= 1 <= s_max, finite
    (the rest shape must lie in the constraint set)."""
    m = I.icosahedron()
    base = I.RBC_MATERIAL.as_tuple() + (0.0, 0.0)
    for ok in ((0.0, 0.0), (1.0, 1.0), (0.9, 1.1), (1.0, 1.5), (0.5, 1.0)):
        native.analyze_cell_type(m.verts, m.tris, base + ok, 0.1)
    for bad in ((1.1, 1.2), (0.8, 0.9), (0.0, 1.1), (-0.1, 1.1), (0.9, float("inf")), (float("nan"), 1.1),
                (1.2, 1.1)):
        with pytest.raises(native.NpfemError, match="strain limits") as ei:
            native.analyze_cell_type(m.verts, m.tris, base + bad, 0.1)
        assert ei.value.code == -1, bad


def test_non_spd_material_is_rejected(lib):
    m = I.rbc_mesh(2)
    _expect(-3, lambda: native.analyze_cell_type(m.verts, m.tris, (-50.0, 0.05, 10, 10, 1.1), 10.0))


def test_last_error_string_is_set(lib):
    try:
        native.analyze_cell_type(I.icosahedron().verts, I.icosahedron().tris[:-1], (1, 1, 1, 1, 1), 0.1)
    except native.NpfemError as e:
        assert "open edge" in str(e) or "closed" in str(e)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets a C compiler
    gives the header's structs (catches a field added on one side only)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"npfem_mesh": native._Mesh, "npfem_material": native._Material,
               "npfem_solver_opts": native._Opts, "npfem_type_info": native._TypeInfo,
               "npfem_collision_params": native._CollisionParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "npfem.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (l.split() for l in out if l)}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_checks_tensors_before_passing_pointers():
    """The Python binding refuses host tensors, wrong dtypes and wrong shapes before any
    pointer reaches the library (checked here on CPU tensors, without a GPU)."""
    torch = pytest.importorskip("torch")
    from paper_2011_04332_b300 import native
    x = torch.zeros(3, 24, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        native._check_step_args(2, 24, native.FP64, x, x, x, None, None, None, None, None)
    with pytest.raises(ValueError, match="required"):
        native._check_step_args(2, 24, native.FP64, None, x, x, None, None, None, None, None)
    a = np.zeros((3, 24), np.float32)
    with pytest.raises(ValueError, match="dtype"):
        native._check_host("x", a, np.float64, (3, 24))
    with pytest.raises(ValueError, match="shape"):
        native._check_host("x", a, np.float32, (3, 25))
    with pytest.raises(ValueError, match="contiguous"):
        native._check_host("x", np.zeros((24, 3), np.float32).T, np.float32, (3, 24))
    native._check_host("status", np.zeros(5, np.int32), np.int32, (5,))
