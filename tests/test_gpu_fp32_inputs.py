"""FP32-storage products on FP32 inputs of every class.

The mixed-precision products widen each gathered FP32 value to FP64 by
integer operations on its encoding (normal numbers) or the conversion
instruction (zeros, subnormals, infinities, NaNs).  These tests
feed x of subnormal floats, signed zeros, and normal floats near the top and
the bottom of the exponent range through every path that widens values --
the factored product (block and single column), the group scan and the
filter/verify scan -- and compare y with the oracle on the exactly widened
inputs.  A wrong exponent or mantissa shift for any class shows up as an
error far above the bound.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

MIXED = 1  # QSD_FP32_MIXED


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_18731_gb300 as q
    c = q.create(0)
    yield c
    c.close()


def _cases():
    h1, eri = wl.chem_integrals(8, seed=8)
    chem = wl.molecular_qubit_operator(h1, eri)
    strings = [v for v in range(1 << 8) if bin(v).count("1") == 4]
    yield "chem", chem, wl.product_subspace(strings, strings, 8), (1, 4, 16)
    yield "xxz", wl.xxz_square(4, 4, 1.0, 0.5), wl.xxz_walk_subspace(4, 4, 3000, seed=2), (1, 16)
    yield "ising", wl.ising_heavy_hex(60, seed=4), wl.flip_subspace(60, 2600, max_flips=3, seed=8), (1,)


def _inputs(rng, shape):
    """float32 arrays: all subnormal; signed zeros among normals; huge and tiny normals."""
    sub = (rng.normal(size=shape) * 2.0 ** -135).astype(np.float32)
    assert np.all(np.abs(sub[sub != 0]) < np.finfo(np.float32).tiny)
    mixed = rng.normal(size=shape).astype(np.float32)
    mixed[rng.random(shape) < 0.3] = 0.0
    mixed[rng.random(shape) < 0.2] = -0.0
    big = (rng.normal(size=shape) * 2.0 ** 100).astype(np.float32)
    small = (rng.normal(size=shape) * 2.0 ** -120).astype(np.float32)
    return {"subnormal": sub, "signed_zeros": mixed, "huge": big, "tiny_normal": small}


@pytest.mark.parametrize("case", ["chem", "xxz", "ising"])
def test_mixed_product_widens_every_float_class(ctx, case):
    import torch
    import paper_2603_18731_gb300 as q
    name, op, words, ks = next(c for c in _cases() if c[0] == case)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    rng = np.random.default_rng(7)
    paths = [0]
    if case == "chem":
        paths = [7]
    elif case == "ising":
        paths = [0, 8]
    for k in ks:
        shape = (sub.dim, k) if k > 1 else (sub.dim,)
        for label, x in _inputs(rng, shape).items():
            ref = oracle.apply(op, keys, x.astype(np.float64)).real
            for path in paths:
                knob = {0: 1, 7: 4, 8: 5}[path]
                ctx.set_tuning(1, knob)
                taken = ctx.product_path(h, sub, MIXED, k)
                assert taken in {0: (0, 1), 7: (7,), 8: (8,)}[path], (case, k, path, taken)
                with torch.cuda.stream(ctx.stream):
                    xd = torch.as_tensor(x, device=ctx.device)
                y = ctx.apply_H(h, sub, xd, precision=MIXED)
                ctx.synchronize()
                got = y.double().cpu().numpy()
                # each row accumulated in FP64 and rounded once to FP32
                # (subnormal results: to a multiple of 2^-149)
                bound = 2.0 ** -22 * float(np.max(np.abs(ref))) + 2.0 ** -148
                err = float(np.max(np.abs(got - ref)))
                assert err <= bound, (case, k, label, path, err, bound)
                if label == "signed_zeros":
                    assert np.all(np.isfinite(got))
    ctx.set_tuning(1, 0)
