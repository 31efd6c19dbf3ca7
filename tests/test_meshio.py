"""Surface-mesh ingestion (PLY, OBJ) on the CPU: generated meshes written to
files and read back give the same connectivity and the same neighbour CSRs
from the oracle; corner forms, relative indices, extra properties, byte
orders and mixed triangle/quad files; refused inputs."""
import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import meshio


def tri_quad_mix():
    el = [(mg.TRI, (0, 1, 4)), (mg.QUAD, (1, 2, 5, 4)), (mg.TRI, (2, 3, 5)), (mg.QUAD, (3, 0, 6, 7))]
    return mg.from_elements(el, 9, "mix")


def quad_first_mix():
    """Mixed, starting with a quad: the binary reader's one-shot read of
    four-corner faces would run past the file and must fall back."""
    el = [(mg.QUAD, (0, 1, 5, 4)), (mg.TRI, (1, 2, 5)), (mg.TRI, (2, 6, 5)), (mg.TRI, (2, 3, 6))]
    return mg.from_elements(el, 7, "quad_first")


MESHES = {"tri40": lambda: mg.tri_grid(40, 3), "tri_holes": lambda: mg.tri_grid(30, 5, holes=0.1),
          "quad20": lambda: mg.quad_grid(20, 4), "mix": tri_quad_mix, "quad_first": quad_first_mix}
WRITERS = {"ply_bin": lambda m, p: meshio.write_ply(m, p), "ply_ascii": lambda m, p: meshio.write_ply(m, p, False),
           "ply_be": lambda m, p: meshio.write_ply(m, p, big_endian=True),
           "ply_extra": lambda m, p: meshio.write_ply(m, p, vertex_extra=("confidence", "intensity")),
           "obj": meshio.write_obj}


def same_mesh(a, b):
    assert a.etype == b.etype and a.n_nodes == b.n_nodes
    np.testing.assert_array_equal(a.conn, b.conn)
    if a.etype == mg.MIXED:
        np.testing.assert_array_equal(a.elem_ptr, b.elem_ptr)
        np.testing.assert_array_equal(a.elem_type, b.elem_type)


@pytest.mark.parametrize("fmt", sorted(WRITERS))
@pytest.mark.parametrize("name", sorted(MESHES))
def test_round_trip(tmp_path, name, fmt):
    m = MESHES[name]()
    path = str(tmp_path / ("m.obj" if fmt == "obj" else "m.ply"))
    WRITERS[fmt](m, path)
    r = meshio.read_mesh(path)
    same_mesh(m, r)
    a, b = oracle.neighbors(m), oracle.neighbors(r)
    for k in ("nodes", "elems"):
        np.testing.assert_array_equal(a[k][0], b[k][0])
        np.testing.assert_array_equal(a[k][1], b[k][1])


def test_obj_corner_forms_and_relative_indices(tmp_path):
    p = tmp_path / "t.obj"
    p.write_text("# a square split in two, with texture and normal indices\n"
                 "v 0 0 0\nv 1 0 0\nv 1 1 0\nv 0 1 0\nvt 0 0\nvn 0 0 1\n"
                 "f 1/1/1 2/1/1 3/1/1\n"
                 "f -4//1 -2//1 -1//1\n"
                 "\n")
    m = meshio.read_obj(str(p))
    assert m.etype == mg.TRI and m.n_nodes == 4
    assert m.conn.tolist() == [0, 1, 2, 0, 2, 3]


def test_ply_with_extra_face_property(tmp_path):
    """A face element with a property after the index list takes the
    per-face path; the list is found by name."""
    p = tmp_path / "f.ply"
    head = ("ply\nformat binary_little_endian 1.0\nelement vertex 4\nproperty float x\nproperty float y\n"
            "property float z\nelement face 2\nproperty list uchar int vertex_indices\nproperty uchar red\n"
            "end_header\n")
    body = np.zeros(12, "<f4").tobytes()
    for nd in ((0, 1, 2), (0, 2, 3)):
        body += bytes([3]) + np.array(nd, "<i4").tobytes() + bytes([200])
    p.write_bytes(head.encode() + body)
    m = meshio.read_ply(str(p))
    assert m.etype == mg.TRI and m.conn.tolist() == [0, 1, 2, 0, 2, 3]


@pytest.mark.parametrize("text,msg", [
    ("v 0 0 0\nv 1 0 0\nv 1 1 0\nv 0 1 0\nv 2 2 0\nf 1 2 3 4 5\n", "5 corners"),
    ("v 0 0 0\nv 1 0 0\nf 1 2 3\n", "does not exist"),
])
def test_obj_refusals(tmp_path, text, msg):
    p = tmp_path / "bad.obj"
    p.write_text(text)
    with pytest.raises(ValueError, match=msg):
        meshio.read_obj(str(p))


def test_ply_refusals(tmp_path):
    p = tmp_path / "bad.ply"
    p.write_bytes(b"solid stl\n")
    with pytest.raises(ValueError, match="not a PLY"):
        meshio.read_ply(str(p))
    p.write_bytes(b"ply\nformat binary_middle_endian 1.0\nend_header\n")
    with pytest.raises(ValueError, match="format"):
        meshio.read_ply(str(p))
    with pytest.raises(ValueError, match="unknown mesh file"):
        meshio.read_mesh(str(tmp_path / "m.stl"))
