"""Bit-exact check of the conversions the kernels do on the integer bits
(to keep them off GB300's narrow FP64 pipe) against the hardware conversions,
through fe_selftest_conversions:

* FP64 -> FP32 round to nearest even: the general integer-bit conversion must
  equal the hardware one for every input (its rare cases call the hardware);
  the branch-free one must equal it wherever it does not raise its
  out-of-range flag, and must raise it wherever the result is not zero or an
  FP32 normal number; the branch-free remainder x - round(x), rounded to FP32,
  likewise;
* an FP32 pair (hi, lo) rounded once to FP64 (the scatter's write-out and the
  cell vectors' fixed-point sum) against one hardware FP64 addition of the
  exactly converted parts;
* FP32 -> FP64 on the integer bits against the hardware conversion;
* the TF32 split of the tensor-core operands against a model of round to
  nearest, ties away from zero, on 10 mantissa bits.

Inputs: random values over 600 binary orders of magnitude, exact halfway
cases of the FP32 rounding (even and odd), results that are FP32 subnormal,
that overflow to infinity or sit at the top of the range, +-0, +-inf, NaN."""
import numpy as np
import pytest
import torch

from paper_1708_01773_gb300 import build, feasm

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(7)
    n = 200_000
    x = [rng.standard_normal(n) * 2.0 ** rng.integers(-300, 300, n)]
    x.append(rng.standard_normal(n) * 2.0 ** rng.integers(-20, 20, n))
    m = rng.integers(1 << 23, 1 << 24, 4000).astype(np.float64)
    e = rng.integers(-100, 100, 4000).astype(np.float64)
    # FP32 halfway cases: 24-bit mantissa + exactly one half unit, and one bit above/below it
    for d in (0.5, 0.5 + 2.0 ** -28, 0.5 - 2.0 ** -28):
        x.append((m + d) * 2.0 ** e)
        x.append(-(m + d) * 2.0 ** e)
    # subnormal FP32 results, the FP32 normal boundary, the top of the range and overflow
    x.append(rng.uniform(1, 2, 4000) * 2.0 ** rng.integers(-152, -124, 4000))
    fmax = float(np.finfo(np.float32).max)
    x.append(fmax * rng.uniform(0.999, 1.001, 4000))
    x.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, 2.0 ** 128, 2.0 ** -126, 2.0 ** -149,
                       2.0 ** -150, 3 * 2.0 ** -151, 1.0, -1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24]))
    return np.concatenate(x)


def _bits32(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def _bits64(a):
    return np.asarray(a, dtype=np.float64).view(np.uint64)


def _same32(a, b):
    a, b = np.asarray(a, np.float32), np.asarray(b, np.float32)
    return (_bits32(a) == _bits32(b)) | (np.isnan(a) & np.isnan(b))


def _tf32_model(f):
    u = _bits32(f).astype(np.uint64)
    r = ((u + 0x1000) & ~np.uint64(0x1fff)).astype(np.uint32)
    return r.view(np.float32)


def test_integer_bit_conversions_match_hardware():
    build.build()
    assert torch.cuda.is_available()
    x = _inputs()
    n = x.size
    xd = torch.tensor(x, device="cuda")
    o32 = torch.empty(n * 8, dtype=torch.float32, device="cuda")
    o64 = torch.empty(n * 5, dtype=torch.float64, device="cuda")
    feasm.fe_selftest_conversions(xd, o32, o64)
    torch.cuda.synchronize()
    o32 = o32.cpu().numpy().reshape(n, 8)
    o64 = o64.cpu().numpy().reshape(n, 5)
    hw, gen, fast, flags, rest, rest_hw, th, tl = o32.T
    flags = flags.astype(np.int32)
    # the hardware rounding itself agrees with numpy's FP64 -> FP32 cast
    with np.errstate(over="ignore"):
        assert _same32(hw, x.astype(np.float32)).all()
    # general conversion: every input
    assert _same32(gen, hw).all()
    # branch-free conversion: exact where unflagged, flagged wherever the
    # result is not zero or FP32-normal
    ok = (flags & 1) == 0
    assert _same32(fast[ok], hw[ok]).all()
    mag = _bits32(hw) & 0x7fffffff
    normal = (mag == 0) | ((mag >= 0x00800000) & (mag < 0x7f800000))
    # (a rounding at the top of the range that carries into infinity is exact
    # unflagged: its value is checked above)
    assert (~ok | normal | (mag == 0x7f800000)).all()
    ordinary = (mag >= 0x00800000) & (mag < 0x7f800000)
    assert ok[ordinary].mean() > 0.99                  # the fast path covers the FP32 normal range
    # branch-free remainder, where unflagged and the rounding is normal
    okr = ok & ((flags & 2) == 0) & normal
    assert _same32(rest[okr], rest_hw[okr]).all()
    # pair -> FP64 rounded once (finite pairs)
    fin = np.isfinite(hw) & np.isfinite(rest_hw)
    p_int, p_fx, p_hw, f_int, f_hw = o64.T
    # (a zero result keeps the sign of hi in the integer path: compared as values)
    zero = p_hw[fin] == 0
    assert ((_bits64(p_int[fin]) == _bits64(p_hw[fin])) | (zero & (p_int[fin] == 0))).all()
    assert ((_bits64(p_fx[fin]) == _bits64(p_hw[fin])) | (zero & (p_fx[fin] == 0))).all()
    # FP32 -> FP64
    same = (_bits64(f_int) == _bits64(f_hw)) | (np.isnan(f_int) & np.isnan(f_hw))
    assert same.all()
    # TF32 split: hi is the model's rounding, lo the rounding of the exact rest,
    # hi + lo within 2^-21 of the FP32 value
    ft = np.isfinite(hw) & (np.abs(hw) < 3.0e38)
    assert _same32(th[ft], _tf32_model(hw[ft])).all()
    assert _same32(tl[ft], _tf32_model((hw[ft] - th[ft]).astype(np.float32))).all()
    # (the split loses the value's low bits only where lo falls below the FP32 normal range)
    big = ft & (np.abs(hw) >= 2.0 ** -100)
    err = np.abs(hw[big].astype(np.float64) - th[big].astype(np.float64) - tl[big].astype(np.float64))
    assert (err <= 2.0 ** -21 * np.abs(hw[big].astype(np.float64))).all()
