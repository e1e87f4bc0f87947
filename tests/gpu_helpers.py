"""Helpers shared by the GPU parity tests (device transfer, oracle references, tolerances).

Tolerances (componentwise error max |got - ref| / sum|terms|, ref and sum|terms|
from the FP64 oracle): FP32 factors 1e-5; BF16 factors 1e-5 against the oracle
on the BF16-rounded factors, and 1e-2 against the oracle on the original FP32
factors (tol_bf16: the BF16 rounding bound where that is larger, orders 4 and 5).
"""
import numpy as np
import pytest

import oracle
import synth

TOL_F32 = 1e-5
TOL_BF16 = 1e-2


def tol_bf16(order):
    """BF16 factors against the oracle on the FP32 factors: 1e-2, or the rounding bound when that is larger.
    Each of a term's order - 1 factor values carries a relative rounding error of at most u = 2^-8 (8-bit
    significand, round to nearest even), so a term is off by at most (1 + u)^(order-1) - 1 of its magnitude:
    7.8e-3 for order 3, 1.18e-2 for order 4, 1.57e-2 for order 5 (reached by output rows with one term)."""
    return max(TOL_BF16, (1.0 + 2.0 ** -8) ** (order - 1) - 1.0 + TOL_F32)

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09266_gb300 as sg
    sg.load()
    return sg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def canonical_split(order, cidx, cval):
    """Oracle canonical entries reordered as strict stream then diagonal stream (order kept)."""
    rows = cidx.T
    eq = (rows[:, 1:] == rows[:, :-1]).any(axis=1) if order > 1 else np.zeros(rows.shape[0], bool)
    strict = ~eq
    o = np.concatenate([np.nonzero(strict)[0], np.nonzero(~strict)[0]])
    return cidx[:, o], cval[o], int(strict.sum())


def factor(n, rank, seed, bf16=False):
    B = synth.factor_normal(n, rank, seed)
    if bf16:
        bits = synth.bf16_rne(B)
        Bt = dev(bits.view(np.int16)).view(torch.bfloat16)
        return Bt, B, synth.bf16_to_f32(bits)
    return dev(B), B, B
