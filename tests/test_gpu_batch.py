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
    # every other mesh scrambled: random vertex ids and cell order, rotated local vertex orders
    probs = [inputs.scrambled(p, seed=30 + i) if i % 2 else p for i, p in enumerate(probs)]
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


def on_tensor_cores(p, prec):
    """fe_assemble's automatic kernel choice: tcgen05 for Q2 elasticity and for
    the BF16 forms of Q3 Poisson and Q3 elasticity ((p+1)^3 rules)."""
    if prec == "fp64" or p.quad_1d != p.order + 1:
        return False
    return (p.order == 2 and p.problem == inputs.ELASTICITY) or (p.order == 3 and prec == "bf16")


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
        # the same arithmetic as a single-space assembly: the tensor-core kernel
        # where fe_assemble's automatic choice takes it, else the CUDA-core one
        s.set_kernel("auto" if on_tensor_cores(p, prec) else "cuda_core")
        sv, sr = s.assemble(torch.tensor(p.coef, device="cuda"), prec=prec)
        s.set_kernel("auto")
        assert torch.equal(sv, vals[i]) and torch.equal(sr, rhs[i]), p.name
    feasm.fe_batch_destroy(batch)


def test_batch_follows_kernel_selection(small_batch):
    """The BF16 batch runs the Q3 spaces' tensor-core cell kernels; after one Q3
    space is switched to the CUDA cores the next call rebuilds its work list with
    that space's cell items and matches the single-space CUDA-core assembly bit
    for bit, and switching back restores the tensor-core result."""
    probs, spaces = small_batch
    i = next(k for k, p in enumerate(probs) if p.order == 3)
    batch = feasm.fe_batch_create([s.handle for s in spaces])
    coef = torch.tensor(probs[i].coef, device="cuda")
    v_tc, _ = batch_run(batch, probs, spaces, "bf16")
    sv, _ = spaces[i].assemble(coef, prec="bf16")
    assert torch.equal(sv, v_tc[i])
    spaces[i].set_kernel("cuda_core")
    v_cc, _ = batch_run(batch, probs, spaces, "bf16")
    sv, _ = spaces[i].assemble(coef, prec="bf16")
    assert torch.equal(sv, v_cc[i]) and not torch.equal(v_cc[i], v_tc[i])
    spaces[i].set_kernel("auto")
    v_back, _ = batch_run(batch, probs, spaces, "bf16")
    assert torch.equal(v_back[i], v_tc[i])
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


def _sampled_rows(n, k=24, seed=0):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, k)])).astype(np.int64)


# orders and problems of the batched recipe at sizes where items hold many cell
# blocks: Q3 elasticity on 20^3 cells (the autotuner's candidates are 1, 4 or 16
# cell blocks per item; a fixed item of 256 cells is compared bit for bit too)
MIX = [((20, 20, 20), 3, 1), ((16, 16, 16), 2, 1), ((24, 24, 24), 1, 0), ((14, 14, 14), 3, 0), ((20, 20, 20), 1, 1),
       ((18, 18, 18), 2, 0)]


@pytest.fixture(scope="module")
def mixed_batch():
    build.build()
    assert torch.cuda.is_available()
    probs = [inputs.small_problem(n, p, pr, seed=600 + i) for i, (n, p, pr) in enumerate(MIX)]
    spaces = [feasm.FESpace(p) for p in probs]
    yield probs, spaces
    for s in spaces:
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16"])
def test_batch_realistic_mix_sampled_rows(mixed_batch, prec):
    probs, spaces = mixed_batch
    auto = feasm.fe_batch_create([s.handle for s in spaces])
    vals, rhs = batch_run(auto, probs, spaces, prec)
    fixed = feasm.fe_batch_create([s.handle for s in spaces], cells_per_item=256)
    vals2, rhs2 = batch_run(fixed, probs, spaces, prec)
    for i, (p, s) in enumerate(zip(probs, spaces)):
        assert torch.equal(vals[i], vals2[i]) and torch.equal(rhs[i], rhs2[i]), p.name
        rows = _sampled_rows(s.n_dofs, seed=i)
        ptr, col_o, val_o, rhs_o = oracle.assemble_rows(p, rows, s.cell_dofs(), s.n_dofs)
        rp, col = s.pattern_host()
        v = vals[i].cpu().numpy()
        worst = 0.0
        for q, r in enumerate(rows):
            np.testing.assert_array_equal(col[rp[r]:rp[r + 1]], col_o[ptr[q]:ptr[q + 1]])
            ref = val_o[ptr[q]:ptr[q + 1]]
            worst = max(worst, np.abs(v[rp[r]:rp[r + 1]] - ref).max() / np.abs(ref).max())
        assert worst <= TOL[prec], (p.name, prec, worst)
        r_gpu = rhs[i].cpu().numpy()[rows]
        assert np.abs(r_gpu - rhs_o).max() <= 1e-12 * max(np.abs(rhs_o).max(), 1e-300), p.name
    feasm.fe_batch_destroy(auto)
    feasm.fe_batch_destroy(fixed)


def test_batch_bounded_wait_runs_out(small_batch):
    """The failure path of the persistent launch: with the test hook, every row item
    waits for one integrated cell more than its space has, gives up after 1e5
    clock cycles, and its block leaves; the launch ends, fe_status reports
    FE_ERR_TIMEOUT for the spaces, and the next normal call on the same batch (same
    captured graph) matches the oracle again. No GPU fault is involved."""
    probs, spaces = small_batch
    batch = feasm.fe_batch_create([s.handle for s in spaces])
    batch_run(batch, probs, spaces, "fp32")                       # tunes and captures
    feasm.fe_batch_set_wait(batch, 100000, 1)
    coefs = [torch.tensor(p.coef, device="cuda") for p in probs]
    vals = [torch.full((s.nnz,), np.nan, dtype=torch.float64, device="cuda") for s in spaces]
    rhs = [torch.full((s.n_dofs,), np.nan, dtype=torch.float64, device="cuda") for s in spaces]
    feasm.fe_batch_assemble(batch, coefs, [p.force for p in probs], vals, rhs, feasm.FE_PREC_FP32)
    torch.cuda.synchronize()
    codes = [s.status() for s in spaces]
    assert all(c == -5 for c in codes), codes                   # FE_ERR_TIMEOUT
    assert all(s.status() == 0 for s in spaces)                  # the words are cleared
    feasm.fe_batch_set_wait(batch, 0, 0)
    vals, rhs = batch_run(batch, probs, spaces, "fp32")
    for i, p in enumerate(probs):
        rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(p)
        assert row_scaled_error(rp_o, col_o, vals[i].cpu().numpy(), val_o) <= TOL["fp32"], p.name
        assert vec_error(rhs[i].cpu().numpy(), rhs_o) <= 1e-12
    with pytest.raises(feasm.FEError):
        feasm.fe_batch_set_wait(batch, -1, 0)
    feasm.fe_batch_destroy(batch)
