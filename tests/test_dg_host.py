"""CPU tests of the DG setup of the C-ABI library (no GPU): the facets and the
CSR pattern of the interior penalty DG space against the oracle's assembly,
also with rotated cell orderings."""
import numpy as np
import pytest

import oracle
from paper_1708_01773_gb300 import feasm, inputs

from test_oracle_pins import rotated_mesh


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1708_01773_gb300 import build
    build.build()


@pytest.mark.parametrize("p,shape,rotate", [(1, (3, 2, 2), False), (2, (2, 3, 2), True), (3, (2, 1, 2), True)])
def test_dg_pattern_and_facets_match_oracle(p, shape, rotate):
    mesh = inputs.small_problem(shape, p, 0, seed=180 + p).mesh
    if rotate:
        mesh = rotated_mesh(mesh, 190 + p)
    g = feasm.DGSpace(mesh, p, host_only=True)
    rp_o, col_o, _, _ = oracle.dg_assemble(mesh, p, 1.0, 5.0)
    rp, col = g.pattern_host()
    np.testing.assert_array_equal(rp, rp_o)
    np.testing.assert_array_equal(col, col_o)
    nx, ny, nz = shape
    assert g.n_interior == (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert g.n_boundary == 2 * (nx * ny + ny * nz + nx * nz)
    plus, minus, pf, mf, bc, bf = g.facets()
    assert np.all(plus < minus)
    cv = mesh.cell_vertices
    for i in range(g.n_interior):
        for cell, f in ((plus[i], pf[i]), (minus[i], mf[i])):
            assert f < 6
        vp = {cv[plus[i]][v] for v in range(8) if (v >> (pf[i] // 2)) & 1 == pf[i] % 2}
        vm = {cv[minus[i]][v] for v in range(8) if (v >> (mf[i] // 2)) & 1 == mf[i] % 2}
        assert vp == vm and len(vp) == 4
    g.close()


def test_dg_twisted_facet_rejected():
    """Two cells whose shared face carries the same four vertices, but with two
    adjacent corners swapped in the second cell: K+'s face corners do not land
    on K-'s by a symmetry of the square, so setup refuses the mesh (the facet
    kernel reads K-'s reference point off that symmetry)."""
    mesh = inputs.small_problem((2, 1, 1), 1, 0, seed=195).mesh
    cv = mesh.cell_vertices.copy()
    cv[1, [0, 2]] = cv[1, [2, 0]]
    twisted = inputs.Mesh(mesh.coords, cv, mesh.shape, mesh.extent)
    with pytest.raises(feasm.FEError, match="symmetry of the square"):
        feasm.DGSpace(twisted, 1, host_only=True)
    # a half-turn of the shared face (diagonal corners swapped) is a symmetry
    cv = mesh.cell_vertices.copy()
    cv[1, [0, 6]] = cv[1, [6, 0]]
    cv[1, [2, 4]] = cv[1, [4, 2]]
    feasm.DGSpace(inputs.Mesh(mesh.coords, cv, mesh.shape, mesh.extent), 1, host_only=True).close()
