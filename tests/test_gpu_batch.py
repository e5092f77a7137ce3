"""GPU tests of the batched persistent driver (fe_batch_*): many spaces of mixed
order, problem and size in one launch, against the oracle and against the
single-space CUDA-core path."""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, energy_error, row_scaled_error, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_batch():
    build.build()
    assert torch.cuda.is_available()
    probs = inputs.batched64(n_meshes=12, n_lo=2, n_hi=5)
    spaces = [feasm.FESpace(p) for p in probs]
    yield probs, spaces
    for s in spaces:
        s.close()


def batch_run(batch, probs, spaces, prec):
    coefs = [torch.tensor(p.coef, device="cuda") for p in probs]
    vals = [torch.full((s.nnz,), np.nan, dtype=torch.float64, device="cuda") for s in spaces]
    rhs = [torch.full((s.n_dofs,), np.nan, dtype=torch.float64, device="cuda") for s in spaces]
    feasm.fe_batch_assemble(batch, coefs, [p.force for p in probs], vals, rhs, feasm.PRECISIONS[prec])
    torch.cuda.synchronize()
    for s in spaces:
        assert s.status() == 0
    return vals, rhs


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16"])
def test_batch_matches_oracle_and_single_space(small_batch, prec):
    probs, spaces = small_batch
    batch = feasm.fe_batch_create([s.handle for s in spaces])
    vals, rhs = batch_run(batch, probs, spaces, prec)
    vals2, rhs2 = batch_run(batch, probs, spaces, prec)          # graph replay, bitwise identical
    for i, (p, s) in enumerate(zip(probs, spaces)):
        assert torch.equal(vals[i], vals2[i]) and torch.equal(rhs[i], rhs2[i])
        rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(p)
        v = vals[i].cpu().numpy()
        assert row_scaled_error(rp_o, col_o, v, val_o) <= TOL[prec], (p.name, prec)
        assert energy_error(rp_o, col_o, v, val_o) <= TOL[prec], (p.name, prec)
        assert vec_error(rhs[i].cpu().numpy(), rhs_o) <= 1e-12
        # the same CUDA-core arithmetic as a single-space assembly
        s.set_kernel("cuda_core")
        sv, sr = s.assemble(torch.tensor(p.coef, device="cuda"), prec=prec)
        s.set_kernel("auto")
        assert torch.equal(sv, vals[i]) and torch.equal(sr, rhs[i]), p.name
    feasm.fe_batch_destroy(batch)


def test_batch_fixed_item_size_and_empty(small_batch):
    probs, spaces = small_batch
    batch = feasm.fe_batch_create([s.handle for s in spaces], cells_per_item=2)
    vals, rhs = batch_run(batch, probs, spaces, "fp32")
    auto = feasm.fe_batch_create([s.handle for s in spaces])
    vals2, rhs2 = batch_run(auto, probs, spaces, "fp32")
    for a, b in zip(vals, vals2):
        assert torch.equal(a, b)
    feasm.fe_batch_destroy(batch)
    feasm.fe_batch_destroy(auto)
    empty = feasm.fe_batch_create([])
    feasm.fe_batch_assemble(empty, [], [], [], [], feasm.FE_PREC_FP32)
    feasm.fe_batch_destroy(empty)
