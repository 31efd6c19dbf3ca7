"""Two GPU paths checked element by element against the oracle.

The paper's own pipeline (Sec. 2.2.1: pairs emitted per element, sorted by
key, reduced by key) run on the GPU with library primitives, as the benchmark
times it -- a comparison, not a code path of the library.  And surface meshes
that went through the PLY and OBJ readers (Sec. 3.1 reads its test models
from such files), built by the library on the GPU."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import meshio, nn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def _check(got, ref):
    for key, (rp, col) in got.items():
        rp = rp.cpu().numpy()
        np.testing.assert_array_equal(rp, ref[key][0], err_msg=f"{key} row_ptr")
        np.testing.assert_array_equal(col.cpu().numpy()[: rp[-1]].astype(np.int32), ref[key][1], err_msg=f"{key} col")


@pytest.mark.parametrize("name,make", [("tri300", lambda: mg.tri_grid(300, 41, holes=0.03)),
                                       ("tet41", lambda: mg.tet_grid(41, 42)),
                                       ("hex61", lambda: mg.hex_grid(61, 43))])
def test_paper_pipeline_on_the_gpu_equals_the_oracle(name, make):
    import torch
    import bench
    mesh = make()
    conn = torch.from_numpy(mesh.conn).cuda().view(mesh.n_elems, -1).to(torch.int64)
    rp_n, col_n, rp_e, col_e = bench.sortpipe_build(torch, conn, mesh.etype, mesh.n_nodes)
    ref = oracle.neighbors(mesh, oracle.BOTH)
    _check({"nodes": (rp_n, col_n), "elems": (rp_e, col_e)}, ref)


@pytest.mark.parametrize("fmt", ["ascii", "binary_little_endian", "binary_big_endian", "obj"])
def test_meshes_read_from_files_build_like_the_generated_ones(tmp_path, fmt):
    mesh = mg.tri_grid(120, 44, holes=0.04)
    path = str(tmp_path / ("m.obj" if fmt == "obj" else "m.ply"))
    if fmt == "obj":
        meshio.write_obj(mesh, path)
    else:
        meshio.write_ply(mesh, path, binary=fmt != "ascii", big_endian=fmt == "binary_big_endian")
    back = meshio.read_mesh(path)
    b = nn.Builder()
    got = b.build(nn.DeviceMesh.from_host(back), nn.WANT_BOTH)
    assert got["status"] == 0
    _check({k: got[k] for k in ("nodes", "elems")}, oracle.neighbors(mesh, oracle.BOTH))


def test_mixed_polygon_file_builds_like_the_oracle(tmp_path):
    """A file of triangles and quads (read as a mixed mesh) against the oracle of the mesh read back."""
    path = tmp_path / "mixed.obj"
    lines = []
    n = 20
    for j in range(n):
        for i in range(n):
            lines.append(f"v {i} {j} 0")
    for j in range(n - 1):
        for i in range(n - 1):
            a, b_, c, d = j * n + i + 1, j * n + i + 2, (j + 1) * n + i + 2, (j + 1) * n + i + 1
            if (i + j) % 3 == 0:
                lines.append(f"f {a} {b_} {c} {d}")
            else:
                lines.append(f"f {a} {b_} {c}")
                lines.append(f"f {a} {c} {d}")
    path.write_text("\n".join(lines) + "\n")
    back = meshio.read_mesh(str(path))
    b = nn.Builder()
    got = b.build(nn.DeviceMesh.from_host(back), nn.WANT_BOTH)
    assert got["status"] == 0
    _check({k: got[k] for k in ("nodes", "elems")}, oracle.neighbors(back, oracle.BOTH))
