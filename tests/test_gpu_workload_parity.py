"""The throughput workload itself against the oracle: 3 species x 256^3 particles on
a 256^3 grid, 200 steps from z = 1e9 to 31, FP32 grids with the FP64 phase-space
state, run as the benchmark runs it (the autotuner's schedule, one recorded CUDA
graph of the whole run).  Particles are independent once the metric is known
(Sec. 2.1), so a random sample of 4096 particles per species, integrated by the
oracle through the same 200 steps (each with its own 256^3 field build), checks
every particle's arithmetic on the full-size path at the method's bars:
positions within 1e-6 L, momenta within 1e-5 relative, weights within 1e-5.

The test also asserts which pass kernel ran: the FP64-state form with its step
integrals evaluated by the fitted polynomials in every pass (fdf_pass_info), the
variant the benchmark times.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_X, TOL_Q, TOL_W = 1e-6, 1e-5, 1e-5
SAMPLE = 4096


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


def test_throughput_workload_sample_matches_the_oracle(F, inputs):
    import torch

    p = inputs.config("c3_3x256")
    tables = inputs.transfer_tables(p)
    stream = torch.cuda.Stream()
    P = F.make_params(p)
    T, keep = F.make_tables(tables)
    P, _, _ = F.fdf_tune(P, T, stream)
    print("schedule:", F.knobs(P))
    n = p["n_part"]
    rng = np.random.default_rng(2024)
    ids = [np.sort(rng.choice(n, SAMPLE, replace=False)) for _ in range(p["n_species"])]
    got = []
    ctx = F.fdf_create(P, T, stream)
    try:
        F.fdf_run_graph(ctx, p["n_steps"])
        info = F.fdf_pass_info(ctx)
        print("pass kernel:", info)
        assert info["form"] == 1 and info["series"] == 1, info
        for s in range(p["n_species"]):
            x = torch.empty((3, n), dtype=torch.float64, device="cuda")
            q = torch.empty((3, n), dtype=torch.float64, device="cuda")
            w = torch.empty((n,), dtype=torch.float64, device="cuda")
            F.fdf_get(ctx, s, x, q, w)
            sel = torch.as_tensor(ids[s], device="cuda")
            got.append((x[:, sel].cpu().numpy(), q[:, sel].cpu().numpy(), w[sel].cpu().numpy()))
            del x, q, w
    finally:
        F.fdf_destroy(ctx)
    gidx = np.concatenate([s * n + ids[s] for s in range(p["n_species"])])
    ref = O.Oracle(p, tables).run(gidx)
    L = p["box"]
    for s in range(p["n_species"]):
        sl = slice(s * SAMPLE, (s + 1) * SAMPLE)
        x, q, w = got[s]
        dx = (x - ref["x"][:, sl] + L / 2) % L - L / 2
        ex = np.max(np.abs(dx)) / L
        eq = np.max(np.linalg.norm(q - ref["q"][:, sl], axis=0) / np.linalg.norm(ref["q"][:, sl], axis=0))
        ew = np.max(np.abs(w - ref["w"][sl]))
        print("species %d: max |dx|/L %.3e  max |dq|/|q| %.3e  max |dw| %.3e" % (s, ex, eq, ew))
        assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (s, ex, eq, ew)
