"""fdf_build_fields_noalloc against the oracle and against fdf_build_fields.

The no-alloc entry point exists for callers that must not allocate device
memory: a simulation code that embeds this library and whose own allocator owns
the whole device budget, or a serving loop that forbids cudaMalloc/cudaFree
after start-up (those calls synchronise the device and fragment its memory).
It runs the same field kernels with their work arrays in one static device
array, so its output must equal the context path's and match the oracle's
fields (or_fields) at the field tolerances of the parity tests.  Two calls in a
row check that the shared array, which keeps the previous call's contents,
does not leak into the next result, and the device's free memory is the same
before and after those calls.  This file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

# the parity tests' field tolerances, relative to each slot's own largest value: FP32
# grids and the FP64 form
TOL = {1: 1e-6, 0: 1e-12}


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


def _err(got, ref):
    return max(np.max(np.abs(got[s] - ref[s])) / np.max(np.abs(ref[s])) for s in range(8))


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_fields_match_the_oracle_and_the_context_path_on_two_calls(F, inputs, c1_tables, prec):
    import torch

    p = inputs.config("c1_32", n_grid=32, precision=prec, seed=31)
    o = O.Oracle(p, c1_tables)
    R = o.noise()
    lnas = [o.lna(37), o.lna(100)]
    oracle = [o.fields(l, 0xFF, R)[0] for l in lnas]
    with F.Run(p, c1_tables) as r:
        context = [r.build_fields(l) for l in lnas]
    P = F.make_params(p)
    T, keep = F.make_tables(c1_tables)
    N = p["n_grid"]
    out = torch.empty((8, N, N, N), dtype=torch.float64, device="cuda")
    # warm-up: the first call looks up the array; torch's fill and copy kernels load their
    # modules on first use, which takes device memory, so they run once here too
    out.fill_(float("nan"))
    F.fdf_build_fields_noalloc(P, T, o.lna(5), out)
    out.cpu()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for lna, ref_o, ref_c in zip(lnas, oracle, context):
        out.fill_(float("nan"))
        F.fdf_build_fields_noalloc(P, T, lna, out)
        got = out.cpu().numpy()
        e_o, e_c = _err(got, ref_o), _err(got, ref_c)
        print("precision %d, ln a %.3f: against the oracle %.3e, against the context path %.3e" % (prec, lna, e_o, e_c))
        assert e_o <= TOL[prec] and e_c <= TOL[prec]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_grids_beyond_the_scratch(F, inputs, c1_tables):
    import torch

    P = F.make_params(inputs.config("c1_32", n_grid=128, precision=1))
    T, keep = F.make_tables(c1_tables)
    out = torch.empty(8 * 128 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FdfError) as e:
        F.fdf_build_fields_noalloc(P, T, -10.0, out)
    assert e.value.code == F.FDF_EINVAL
    assert "FDF_NOALLOC_SCRATCH_BYTES" in F.fdf_last_error()
