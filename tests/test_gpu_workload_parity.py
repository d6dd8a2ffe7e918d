"""The measured workloads themselves against the oracle, run as the benchmark runs
them (the autotuner's schedule for the throughput workload, also applied to the
reduced-precision one; one recorded CUDA graph of the whole run):

* 3 species x 256^3 particles on a 256^3 grid, 200 steps from z = 1e9 to 31,
  FP32 grids with the FP64 phase-space state;
* 512^3 particles on a 256^3 grid, 300 steps, BF16 grids with the FP64 state.

Particles are independent once the metric is known (Sec. 2.1), so a random
sample of 4096 particles per species, integrated by the oracle through the same
steps (each with its own 256^3 field build), checks the full-size path at the
method's bars: positions within 1e-6 L, momenta within 1e-5 relative, weights
within 1e-5 (the BF16 bars of test_gpu_parity.py for BF16 grids).

The test also asserts which pass kernel ran: the FP64-state form with its step
integrals evaluated by the fitted polynomials in every pass (fdf_pass_info), the
variant the benchmark times.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BARS = {"c3_3x256": (1e-6, 1e-5, 1e-5), "c4_512_bf16": (2e-5, 2.5e-4, 2.5e-4)}
SAMPLE = 4096


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


@pytest.fixture(scope="module")
def schedule(F, inputs):
    """The autotuner's knobs for the throughput workload (as bench.py takes them)."""
    import torch

    p = inputs.config("c3_3x256")
    P = F.make_params(p)
    T, keep = F.make_tables(inputs.transfer_tables(p))
    P, _, _ = F.fdf_tune(P, T, torch.cuda.Stream())
    return F.knobs(P)


@pytest.mark.parametrize("name", ["c3_3x256", "c4_512_bf16"])
def test_workload_sample_matches_the_oracle(F, inputs, schedule, name):
    import torch

    p = inputs.config(name)
    tables = inputs.transfer_tables(p)
    P = F.make_params(p)
    for k, v in schedule.items():
        if k != "n_gl":
            setattr(P, k, v)
    T, keep = F.make_tables(tables)
    print("%s schedule: %s" % (name, F.knobs(P)))
    n = p["n_part"]
    rng = np.random.default_rng(2024)
    ids = [np.sort(rng.choice(n, SAMPLE, replace=False)) for _ in range(p["n_species"])]
    got = []
    ctx = F.fdf_create(P, T, torch.cuda.Stream())
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
    bx, bq, bw = BARS[name]
    for s in range(p["n_species"]):
        sl = slice(s * SAMPLE, (s + 1) * SAMPLE)
        x, q, w = got[s]
        dx = (x - ref["x"][:, sl] + L / 2) % L - L / 2
        ex = np.max(np.abs(dx)) / L
        eq = np.max(np.linalg.norm(q - ref["q"][:, sl], axis=0) / np.linalg.norm(ref["q"][:, sl], axis=0))
        ew = np.max(np.abs(w - ref["w"][sl]))
        print("%s species %d: max |dx|/L %.3e  max |dq|/|q| %.3e  max |dw| %.3e" % (name, s, ex, eq, ew))
        assert ex < bx and eq < bq and ew < bw, (s, ex, eq, ew)
