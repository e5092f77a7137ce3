"""Accuracy of the mixed forms over every entry of the full-size workloads.

The FP32 (3xTF32 on the tensor cores for Q2 elasticity, CUDA cores for the
others) and BF16 (tensor cores for Q2 elasticity and the Q3 elements) forms
of the automatic kernel choice are compared over all nonzeros with the FP64 GPU path of the same space,
which the parity tests pin to the oracle on sampled rows (within 1e-14). Row-
scaled entry error (max_ij |a - a*| / max_j |a*_ij|) and energy error
(|v^T (A - A*) v| / v^T A* v over seeded unit-RMS vectors) must stay within the
stated tolerances: 1e-6 (FP32) and 1e-2 (BF16)."""
import pytest
import torch

from metrics import TOL
from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


def _errors(rp, col, vals, ref, n_vec=4, seed=0):
    n = rp.numel() - 1
    rows = torch.repeat_interleave(torch.arange(n, device=rp.device), rp[1:] - rp[:-1])
    rowmax = torch.zeros(n, dtype=torch.float64, device=rp.device)
    rowmax.scatter_reduce_(0, rows, ref.abs(), reduce="amax")
    entry = float(((vals - ref).abs() / rowmax[rows].clamp_min(1e-300)).max())
    del rows, rowmax
    g = torch.Generator(device="cuda").manual_seed(seed)
    D = torch.sparse_csr_tensor(rp, col.to(torch.int64), vals - ref, size=(n, n))
    A = torch.sparse_csr_tensor(rp, col.to(torch.int64), ref, size=(n, n))
    energy = 0.0
    for _ in range(n_vec):
        v = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        energy = max(energy, float(torch.dot(v, torch.mv(D, v)).abs() / torch.dot(v, torch.mv(A, v))))
    return entry, energy


@pytest.mark.parametrize("workload", ["elasticity_q2_beam", "elasticity_q1_128", "poisson_q3_40", "elasticity_q3_20"])
def test_mixed_forms_every_entry_full_size(workload):
    prob = inputs.WORKLOADS[workload]()
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device="cuda")
    ref, rhs_ref = sp.assemble(coef, prec="fp64")
    rp, col = sp.pattern()
    for prec in ("fp32", "bf16"):
        vals, rhs = sp.assemble(coef, prec=prec)
        torch.cuda.synchronize()
        assert sp.status() == 0
        entry, energy = _errors(rp, col, vals, ref)
        print(f"{workload} {prec}: entry {entry:.3e} energy {energy:.3e}")
        assert entry <= TOL[prec], (prec, entry)
        assert energy <= TOL[prec], (prec, energy)
        assert float((rhs - rhs_ref).abs().max() / rhs_ref.abs().max()) <= 1e-12
        del vals, rhs
    sp.close()
