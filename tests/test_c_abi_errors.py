"""Error behaviour of the C ABI, checked without a GPU: invalid arguments and
meshes are rejected with VEM_EINVAL and a message before any device work,
and a valid problem on a machine without a GPU fails with a status instead of
running anywhere else (the library has no CPU path)."""
import ctypes

import numpy as np
import pytest

from synth import cube_mesh

VEM_EINVAL = -1


@pytest.fixture(scope="module")
def pkg():
    import paper_2304_09770_gb300 as p
    p.lib()
    return p


def _assemble(pkg, mesh, k=2, nu=None):
    L = pkg.lib()
    keep = dict(xyz=np.ascontiguousarray(mesh["xyz"], dtype=np.float64),
                fp=np.ascontiguousarray(mesh["face_ptr"], dtype=np.int32),
                fv=np.ascontiguousarray(mesh["face_vtx"], dtype=np.int32),
                ep=np.ascontiguousarray(mesh["elem_ptr"], dtype=np.int32),
                ef=np.ascontiguousarray(mesh["elem_face"], dtype=np.int32))
    i32 = ctypes.POINTER(ctypes.c_int32)
    m = pkg._Mesh(len(keep["xyz"]), keep["xyz"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  len(keep["fp"]) - 1, keep["fp"].ctypes.data_as(i32), keep["fv"].ctypes.data_as(i32),
                  len(keep["ep"]) - 1, keep["ep"].ctypes.data_as(i32), keep["ef"].ctypes.data_as(i32))
    nu = np.ones(len(keep["ep"]) - 1) if nu is None else nu
    h = ctypes.c_void_p()
    st = L.vem_assemble(ctypes.byref(m), int(k), nu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        ctypes.byref(h))
    return st, L.vem_last_error().decode(), h


def _mesh():
    return {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in cube_mesh(2).items()}


def test_null_arguments(pkg):
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.vem_assemble(None, 2, None, ctypes.byref(h)) == VEM_EINVAL
    assert L.bddc_setup(None, None, 15, 1, None, ctypes.byref(h)) == VEM_EINVAL
    assert L.bddc_apply(None, None, None) == VEM_EINVAL
    assert L.vem_apply(None, None, None) == VEM_EINVAL
    assert L.vem_load_noalloc(None, 2, None, None) == VEM_EINVAL
    it, ka, l0, l1 = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    assert L.pcg_solve(None, None, None, 1e-8, 10, ctypes.byref(it), ctypes.byref(ka), ctypes.byref(l0),
                       ctypes.byref(l1)) == VEM_EINVAL
    assert L.vem_last_error().decode()


def test_invalid_degree(pkg):
    st, msg, _ = _assemble(pkg, _mesh(), k=5)
    assert st == VEM_EINVAL and "degree" in msg


@pytest.mark.parametrize("defect", ["vertex_range", "short_face", "zero_face_ref", "face_in_three"])
def test_invalid_meshes(pkg, defect):
    m = _mesh()
    if defect == "vertex_range":
        m["face_vtx"][0] = len(m["xyz"]) + 5
    elif defect == "short_face":
        # drop the last vertex of the first face: a face of 3 -> fine, so make it 2
        fp, fv = m["face_ptr"], m["face_vtx"]
        keep = np.ones(len(fv), dtype=bool)
        keep[fp[0] + 2:fp[1]] = False
        m["face_vtx"] = fv[keep]
        m["face_ptr"] = np.concatenate([[0], fp[1:] - (fp[1] - fp[0] - 2)]).astype(np.int32)
    elif defect == "zero_face_ref":
        m["elem_face"][0] = 0
    elif defect == "face_in_three":
        ef = m["elem_face"]
        ef[m["elem_ptr"][1]] = ef[0]     # element 1 also claims element 0's first face
        ef[m["elem_ptr"][2]] = ef[0]     # and element 2
    st, msg, _ = _assemble(pkg, m)
    assert st == VEM_EINVAL, msg
    assert msg


def test_no_cpu_path_without_a_gpu(pkg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the call would succeed")
    st, msg, h = _assemble(pkg, _mesh())
    assert st != 0, "the library assembled a system without a GPU"
    assert "cuda" in msg.lower() or "device" in msg.lower()


def _prism(m):
    """One prism over a regular m-gon (faces: two m-gons, m quadrilaterals)."""
    a = 2 * np.pi * np.arange(m) / m
    ring = np.stack([0.5 + 0.4 * np.cos(a), 0.5 + 0.4 * np.sin(a)], 1)
    xyz = np.concatenate([np.c_[ring, np.zeros(m)], np.c_[ring, np.ones(m)]])
    faces = [list(range(m))[::-1], list(range(m, 2 * m))]
    faces += [[i, (i + 1) % m, m + (i + 1) % m, m + i] for i in range(m)]
    return {"xyz": xyz, "face_ptr": np.cumsum([0] + [len(f) for f in faces]).astype(np.int32),
            "face_vtx": np.array([v for f in faces for v in f], dtype=np.int32),
            "elem_ptr": np.array([0, len(faces)], dtype=np.int32),
            "elem_face": np.arange(1, len(faces) + 1, dtype=np.int32)}


def test_faces_beyond_the_element_records_are_rejected(pkg):
    """A face with more vertices than an element record holds (12) is
    rejected on the host, before any device work."""
    st, msg, _ = _assemble(pkg, _prism(13))
    assert st == VEM_EINVAL and "vertex count" in msg, msg


def test_cvt_mesh_passes_the_host_checks(pkg):
    """Voronoi cells (up to about 30 vertices, 17 faces, faces of up to 9
    vertices) fit the element records: without a GPU the call gets past
    every host check and fails only at the first device call."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the call would succeed")
    from synth.mesh import cvt_mesh
    st, msg, _ = _assemble(pkg, cvt_mesh(27, seed=5, iters=20))
    assert st != VEM_EINVAL and ("cuda" in msg.lower() or "device" in msg.lower()), msg


def test_reduced_entry_point_checks_its_arguments(pkg):
    h = ctypes.c_void_p()
    assert pkg.lib().vem_assemble_reduced(None, 2, None, ctypes.byref(h)) == VEM_EINVAL


def test_octa_mesh_passes_the_host_checks(pkg):
    """OCTA elements (truncated cubes with pentagons, octahedra) fit the
    element records: on a machine without a GPU the call gets past every
    host check and fails only at the first device call."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the call would succeed")
    from synth.mesh import octa_mesh
    st, msg, _ = _assemble(pkg, octa_mesh(2))
    assert st != VEM_EINVAL and ("cuda" in msg.lower() or "device" in msg.lower()), msg
