"""GPU parity of the Q1 elasticity cell kernel with warp roles (FP32 and BF16
forms, chosen by the automatic kernel selection): FP64 geometry of whole tiles
of 32 cells on their own warps, contraction on the others.

A 41 x 37 x 33 mesh (50,061 cells: more 32-cell tiles than blocks, so every
persistent block loops over tiles and reuses its geometry slots, and a ragged
last tile of 13 cells) is compared with the oracle entry by entry, together with
the general CUDA-core kernel on the same space; small meshes cover a single
partial tile."""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, energy_error, row_scaled_error, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


def _assemble(sp, prob, prec):
    coef = torch.tensor(prob.coef, device="cuda")
    vals, rhs = sp.assemble(coef, prec=prec)
    torch.cuda.synchronize()
    assert sp.status() == 0
    return vals, rhs


@pytest.mark.parametrize("shape", [(41, 37, 33), (3, 2, 2), (1, 1, 1)])
def test_q1_elasticity_warp_roles_every_entry(shape):
    prob = inputs.small_problem(shape, 1, 1, seed=1000 + shape[0])
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob)
    sp = feasm.FESpace(prob)
    for prec in ("fp32", "bf16"):
        sp.set_kernel("auto")
        vals, rhs = _assemble(sp, prob, prec)
        v = vals.cpu().numpy()
        assert row_scaled_error(rp_o, col_o, v, val_o) <= TOL[prec], prec
        assert energy_error(rp_o, col_o, v, val_o) <= TOL[prec], prec
        assert vec_error(rhs.cpu().numpy(), rhs_o) <= 1e-12
        again, rhs2 = _assemble(sp, prob, prec)
        assert torch.equal(vals, again) and torch.equal(rhs, rhs2)      # bitwise reproducible
        sp.set_kernel("cuda_core")                                       # the general path, same space
        vg, rg = _assemble(sp, prob, prec)
        assert row_scaled_error(rp_o, col_o, vg.cpu().numpy(), val_o) <= TOL[prec], prec
        assert vec_error(rg.cpu().numpy(), rhs_o) <= 1e-12
    sp.set_kernel("auto")
    sp.close()


def test_q1_elasticity_warp_roles_negative_jacobian():
    """An inverted cell sets FE_ERR_NEG_JACOBIAN in the warp-role cell kernel too."""
    prob = inputs.small_problem((2, 2, 2), 1, 1, seed=1)
    coords = prob.mesh.coords.copy()
    coords[13] = [1.2, 1.2, 1.2]
    m = inputs.Mesh(coords, prob.mesh.cell_vertices, prob.mesh.shape, prob.mesh.extent)
    bad = inputs.Problem("bad", m, 1, 2, 1, prob.coef, prob.force)
    sp = feasm.FESpace(bad)
    sp.assemble(torch.tensor(bad.coef, device="cuda"), prec="fp32")
    assert sp.status() == -4
    assert sp.status() == 0
    sp.close()
