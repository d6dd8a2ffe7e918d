"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle on the
same seeded inputs.

Bars (from the method's accuracy contract): sampled positions and momenta
bit-exact; final positions within 1e-6 L (periodic distance), momenta within
1e-5 relative per particle, delta-f weights within 1e-5 absolute; density
deposit within 1e-5 relative in the L2 norm.  The plain FP64 form is held to
1e-9 as well, since it differs from the oracle only by rounding and by the
4-node versus 16-node quadrature of the step integrals.

Precision settings (include/fdf.h): 0 plain FP64; 1 FP32 grids with an FP64
phase-space state (FP64 x and q, FP64 step integrals, FP32 kicks); 2 the same
with BF16 grids; 3 and 4 the split-state forms (fixed-point positions, FP32
q_0 + dq) with FP32 and BF16 grids.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL_X, TOL_Q, TOL_W = 1e-6, 1e-5, 1e-5


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


def pdiff(a, b, L):
    return (a - b + L / 2) % L - L / 2


def errors(x, q, w, ref, L):
    ex = np.max(np.abs(pdiff(x, ref["x"], L))) / L if x.size else 0.0
    eq = np.max(np.linalg.norm(q - ref["q"], axis=0) / np.linalg.norm(ref["q"], axis=0)) if q.size else 0.0
    ew = np.max(np.abs(w - ref["w"])) if w.size else 0.0
    return ex, eq, ew


def run_gpu(F, p, tables, steps=None, frozen=None):
    with F.Run(p, tables) as r:
        if frozen is not None:
            r.set_fields(frozen)
        r.sample()
        r.step(p["n_steps"] if steps is None else steps)
        out = [r.get(s) for s in range(p.get("n_species", 1))]
        dep = r.deposit(-1)
    return out, dep


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1, 3])
def test_sampler_bit_exact(F, inputs, c1_tables, prec):
    p = inputs.config("c1_32", n_part=5003, n_species=2, m_ev=[0.05, 0.2], precision=prec, seed=123456789012)
    with F.Run(p, c1_tables) as r:
        r.sample()
        got = [r.get_initial(s) for s in range(2)]
    o = O.Oracle(p, c1_tables)
    for s in range(2):
        X, qs, pm = o.sample(np.arange(s * p["n_part"], (s + 1) * p["n_part"]))
        assert np.array_equal(got[s][0], X)
        assert np.array_equal(got[s][1].view(np.uint64), qs.view(np.uint64))
        assert np.array_equal(got[s][2].view(np.uint64), pm.view(np.uint64))


# The grid bars, each slot's error relative to that slot's own largest value: FP32 and
# FP64 from the method's contract (1e-6 and 1e-12); BF16 from its storage rounding (2^-9).
FIELD_TOL = {0: 1e-12, 1: 1e-6, 2: 4e-3}


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_fields_match_oracle(F, inputs, c1_tables, prec):
    """Each slot against the oracle, on its own scale, at four scale factors from z = 1e9
    to the end.  Slots are transformed in packed pairs (d_x psi + i d_y psi,
    d_z psi + i d_x phi, d_y phi + i d_z phi, phi_dot + i slot 7) and an FFT's rounding is
    relative to the complex signal it transforms: the steps' grids carry zero in slot 7,
    so phi_dot, about 1e4 times smaller than psi late in the run, is transformed alone."""
    tol = FIELD_TOL[prec]
    p = inputs.config("c1_32", n_grid=32, precision=prec, seed=31)
    o = O.Oracle(p, c1_tables)
    R = o.noise()
    errs = []
    with F.Run(p, c1_tables) as r:
        for k in (0, 37, 80, 100):
            lna = o.lna(k)
            g = r.build_fields(lna)
            ref, _ = o.fields(lna, 0xFF, R)
            for s in range(8):
                scale = np.max(np.abs(ref[s]))
                errs.append((k, s, scale, np.max(np.abs(g[s] - ref[s])) / scale))
    for e in errs:
        print("k %3d slot %d  max|ref| %.3e  err / own scale %.3e" % e)
    assert all(e[2] > 0 and e[3] < tol for e in errs)


@pytest.mark.parametrize("prec,N", [(1, 8), (1, 16), (1, 64), (1, 128), (1, 256), (0, 8), (0, 64), (0, 128),
                                    (2, 128)])
def test_fields_match_oracle_at_every_grid_size(F, inputs, c1_tables, prec, N):
    """The FFT passes are compiled per grid size (each N = N1 N2 has its own register
    split and shared-memory shape), so every size the workloads use is checked against
    the oracle, slot by slot on its own scale, at one scale factor in the matter era."""
    p = inputs.config("c1_32", n_grid=N, box=1000.0 * N / 32, precision=prec, seed=33)
    o = O.Oracle(p, c1_tables)
    lna = o.lna(80)
    with F.Run(p, c1_tables) as r:
        g = r.build_fields(lna)
    ref, _ = o.fields(lna, 0xFF, o.noise())
    worst = 0.0
    for s in range(8):
        worst = max(worst, np.max(np.abs(g[s] - ref[s])) / np.max(np.abs(ref[s])))
    print("N %d prec %d: largest slot error / own scale %.3e" % (N, prec, worst))
    assert worst < FIELD_TOL[prec]


def test_run_c1_plain_fp64(F, inputs, c1_tables):
    """The full first workload: 32^3 particles, 32^3 grid, 100 steps, all FP64."""
    p = inputs.config("c1_32")
    (res,), dep = run_gpu(F, p, c1_tables)
    o = O.Oracle(p, c1_tables)
    ref = o.run(np.arange(p["n_part"]))
    ex, eq, ew = errors(*res, ref, p["box"])
    assert ex < 1e-9 and eq < 1e-9 and ew < 1e-10, (ex, eq, ew)
    a = math.exp(o.lna(p["n_steps"]))
    dref = o.deposit(np.arange(p["n_part"]), ref["x"], ref["q"], ref["w"], a, 0)
    assert np.linalg.norm(dep - dref) / np.linalg.norm(dref) < 1e-8


# BF16 storage rounds every field value to 2^-9 relative.  Each kick, and so the
# momentum, carries at most that fraction of the kicks it received; these
# workloads kick a particle by at most ~3% of |q| in total (oracle), so the
# momentum error stays below 2^-9 * 0.03 * (a factor 4 for the trilinear mix and
# correlated roundings) = 2.5e-4, and positions follow with the time integral.
BF16_TOL_X, BF16_TOL_Q, BF16_TOL_W = 2e-5, 2.5e-4, 2.5e-4


@pytest.mark.parametrize("prec,n_steps", [(1, 100), (1, 200), (2, 100), (3, 100), (4, 100)])
def test_run_c1_shapes_fp32_grid_forms(F, inputs, c1_tables, prec, n_steps):
    """The first workload's shapes in the FP32/BF16-grid forms.  With 200 steps the
    FP64-state form evaluates its step integrals with the fitted polynomials (the
    throughput workloads' steps); with 100 the polynomials miss their 2e-13 bar and the
    integrals are summed node by node: both paths are checked."""
    p = inputs.config("c1_32", precision=prec, n_steps=n_steps)
    (res,), dep = run_gpu(F, p, c1_tables)
    o = O.Oracle(p, c1_tables)
    ref = o.run(np.arange(p["n_part"]))
    ex, eq, ew = errors(*res, ref, p["box"])
    print("prec %d, %d steps: max |dx|/L %.3e  max |dq|/q %.3e  max |dw| %.3e" % (prec, n_steps, ex, eq, ew))
    if prec in (2, 4):
        assert ex < BF16_TOL_X and eq < BF16_TOL_Q and ew < BF16_TOL_W, (ex, eq, ew)
        return
    assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)
    a = math.exp(o.lna(p["n_steps"]))
    dref = o.deposit(np.arange(p["n_part"]), ref["x"], ref["q"], ref["w"], a, 0)
    assert np.linalg.norm(dep - dref) / np.linalg.norm(dref) < 1e-5


@pytest.mark.parametrize("prec,spp", [(1, 6), (1, 8), (3, 8)])
def test_long_passes_match_the_oracle(F, inputs, c1_tables, prec, spp):
    """Passes of 6 and 8 leapfrog steps (the longest the launch carries) against the oracle,
    200 steps (the fitted-polynomial path of the FP64-state form)."""
    p = inputs.config("c1_32", n_part=4096, precision=prec, n_steps=200, steps_per_pass=spp)
    (res,), dep = run_gpu(F, p, c1_tables)
    o = O.Oracle(p, c1_tables)
    ref = o.run(np.arange(p["n_part"]))
    ex, eq, ew = errors(*res, ref, p["box"])
    print("prec %d, %d steps per pass: max |dx|/L %.3e  max |dq|/q %.3e  max |dw| %.3e" % (prec, spp, ex, eq, ew))
    assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_ragged_two_species(F, inputs, c1_tables, prec):
    p = inputs.config("c1_32", n_part=3001, n_species=2, m_ev=[0.05, 0.25], n_grid=16, n_steps=40,
                      precision=prec, seed=77)
    res, dep = run_gpu(F, p, c1_tables)
    o = O.Oracle(p, c1_tables)
    for s in range(2):
        ref = o.run(np.arange(s * p["n_part"], (s + 1) * p["n_part"]))
        ex, eq, ew = errors(*res[s], ref, p["box"])
        assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (s, ex, eq, ew)


def test_empty_run(F, inputs, c1_tables):
    p = inputs.config("c1_32", n_part=0, n_grid=8, n_steps=3, precision=1)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(3)
        x, q, w = r.get(0)
        assert x.size == 0
        assert np.all(r.deposit() == 0)


def test_call_order_and_range_errors(F, inputs, c1_tables):
    p = inputs.config("c1_32", n_part=100, n_grid=8, n_steps=5, precision=1)
    with F.Run(p, c1_tables) as r:
        with pytest.raises(F.FdfError) as e:
            r.step(1)
        assert e.value.code == F.FDF_ESTATE
        r.sample()
        with pytest.raises(F.FdfError) as e:
            r.step(6)
        assert e.value.code == F.FDF_EINVAL
        with pytest.raises(F.FdfError) as e:
            r.step(-1)
        assert e.value.code == F.FDF_EINVAL
        r.step(5)
        assert r.state()[0] == 5
        with pytest.raises(F.FdfError) as e:
            r.get_initial(0)
        assert e.value.code == F.FDF_ESTATE


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_zero_potentials(F, inputs, c1_tables, prec):
    p = inputs.config("c1_32", n_part=2000, n_grid=16, n_steps=30, precision=prec)
    z = inputs.zero_tables(c1_tables)
    with F.Run(p, z) as r:
        r.sample()
        X, qs, pm = r.get_initial(0)
        r.step(30)
        x, q, w = r.get(0)
    if prec in (0, 1):
        # FP64 momenta: a kick of exactly zero leaves them bitwise unchanged
        assert np.array_equal(q, qs)
        assert np.all(w == 0.0)
    else:
        assert np.max(np.abs(q - qs) / pm) < 2 ** -46
        assert np.max(np.abs(w)) < 1e-12
    ref = O.Oracle(p, z).run(np.arange(p["n_part"]))
    ex, _, _ = errors(x, q, w, ref, p["box"])
    print("prec %d: max |dx|/L %.3e" % (prec, ex))
    assert ex < {0: 1e-12, 1: 1e-11, 3: 1e-8}[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_uniform_gradient_fields(F, inputs, c1_tables, prec):
    p = inputs.config("c1_32", n_part=1500, n_grid=16, n_steps=30, m_ev=[0.05], precision=prec)
    fr = inputs.uniform_fields(16, [2e-6, -1e-6, 5e-7], [-3e-7, 4e-7, 1e-6], 3e-9, 2e-5)
    (res,), _ = run_gpu(F, p, c1_tables, frozen=fr)
    ref = O.Oracle(p, c1_tables).run(np.arange(p["n_part"]), frozen=fr)
    ex, eq, ew = errors(*res, ref, p["box"])
    print("prec %d: max |dx|/L %.3e  max |dq|/q %.3e  max |dw| %.3e" % (prec, ex, eq, ew))
    if prec in (2, 4):
        assert ex < BF16_TOL_X and eq < BF16_TOL_Q and ew < BF16_TOL_W, (ex, eq, ew)
        return
    # FP64-state form: FP32 kicks (2^-24 of kicks that sum to a few % of |q|) on FP64 state
    bq, bx = {0: (1e-9, 1e-9), 1: (1e-7, 1e-8), 3: (TOL_Q, TOL_X)}[prec]
    assert eq < bq and ex < bx and ew < TOL_W, (ex, eq, ew)


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_reversibility(F, inputs, c1_tables, prec):
    p = inputs.config("c1_32", n_part=4000, n_grid=16, n_steps=60, m_ev=[0.1], precision=prec)
    fr = inputs.cosine_fields(16, p["box"], 3e-4, (1, 2, 3))
    with F.Run(p, c1_tables) as r:
        r.set_fields(fr)
        r.sample()
        r.step(35)
        x0, q0, _ = r.get(0)
        r.step(25)
        x1, q1, _ = r.get(0)
        r.step(-25)
        x2, q2, _ = r.get(0)
    assert np.max(np.linalg.norm(q1 - q0, axis=0) / np.linalg.norm(q0, axis=0)) > 1e-3
    L = p["box"]
    print("prec %d: back-and-forth |dx|/L %.3e |dq|/q %.3e" % (
        prec, np.max(np.abs(pdiff(x2, x0, L))) / L, np.max(np.linalg.norm(q2 - q0, axis=0) / np.linalg.norm(q0, axis=0))))
    # FP64: round-off only.  FP32-grid forms: the FP32 kick sums of the forward and
    # backward passes round differently (2^-24 of each kick, kicks up to a few % of
    # |q|); the split-state form also quantises positions to L / 2^32.
    tol = 1e-12 if prec == 0 else 1e-7
    assert np.max(np.abs(pdiff(x2, x0, L))) < tol * L
    assert np.max(np.linalg.norm(q2 - q0, axis=0) / np.linalg.norm(q0, axis=0)) < tol


@pytest.mark.parametrize("prec", [1, 3])
def test_split_calls_equal_one_call(F, inputs, c1_tables, prec):
    """Stepping 60 then 40 equals stepping 100 (merged versus split half kicks)."""
    p = inputs.config("c1_32", n_part=3000, n_grid=16, precision=prec)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(100)
        a = r.get(0)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(60)
        r.step(40)
        b = r.get(0)
    L = p["box"]
    ex = np.max(np.abs(pdiff(a[0], b[0], L))) / L
    eq = np.max(np.abs(a[1] - b[1]) / np.linalg.norm(a[1], axis=0))
    print("merged vs split kicks: |dx|/L %.3e |dq|/q %.3e" % (ex, eq))
    assert ex < 1e-8 and eq < 1e-9


# ---- the measured workloads at full size (sampled outputs) ---------------------------------------
@pytest.mark.slow
def test_c2_full_size_subset(F, inputs):
    p = inputs.config("c2_128")
    tables = inputs.transfer_tables(p)
    (res,), dep = run_gpu(F, p, tables)
    ids = np.random.default_rng(0).choice(p["n_part"], 4096, replace=False)
    ids.sort()
    ref = O.Oracle(p, tables).run(ids)
    x, q, w = (a[..., ids] for a in res)
    ex, eq, ew = errors(x, q, w, ref, p["box"])
    print("c2: max |dx|/L %.3e  max |dq|/q %.3e  max |dw| %.3e" % (ex, eq, ew))
    assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["c3_3x256", "c4_512_bf16"])
def test_full_size_workloads_few_steps(F, inputs, name):
    """Full particle count and grid of the throughput workloads, the same launch
    shapes as the benchmark, over 10 large steps of the same redshift range;
    a sample of particles of every species is checked against the oracle."""
    p = inputs.config(name, n_steps=10)
    tables = inputs.transfer_tables(p)
    res, _ = run_gpu(F, p, tables)
    o = O.Oracle(p, tables)
    rng = np.random.default_rng(1)
    for s in range(p["n_species"]):
        ids = np.sort(rng.choice(p["n_part"], 512, replace=False))
        ref = o.run(s * p["n_part"] + ids)
        x, q, w = (a[..., ids] for a in res[s])
        ex, eq, ew = errors(x, q, w, ref, p["box"])
        print("%s species %d: max |dx|/L %.3e  max |dq|/q %.3e  max |dw| %.3e" % (name, s, ex, eq, ew))
        if p["precision"] == 2:
            assert ex < BF16_TOL_X and eq < BF16_TOL_Q and ew < BF16_TOL_W, (ex, eq, ew)
        else:
            assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)


@pytest.mark.parametrize("n_steps", [200, 100])
def test_pass_shapes_give_identical_results(F, inputs, c1_tables, n_steps):
    """The FP64-state pass's launch shapes (pass_blocks 1, 2, 3: with two blocks per SM each
    thread carries two particles in lockstep) run the same arithmetic per particle: the
    results are bitwise equal.  Two ragged species, so that chunks end part-way and a
    thread's second particle can fall past the end."""
    p = inputs.config("c1_32", n_part=3001, n_species=2, m_ev=[0.05, 0.2], n_grid=16, n_steps=n_steps,
                      precision=1, seed=91)
    got = {}
    for pb in (1, 2, 3):
        with F.Run(dict(p, pass_blocks=pb), c1_tables) as r:
            r.sample()
            r.step(n_steps)
            got[pb] = [r.get(s) for s in range(2)]
    for pb in (1, 2):
        for s in range(2):
            for a, b in zip(got[pb][s], got[3][s]):
                assert np.array_equal(a, b), (pb, s)


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_get_into_page_locked_host_memory(F, inputs, c1_tables, prec):
    """fdf_get into page-locked host buffers (written by the device directly), into
    pageable host buffers (through the staging buffer) and into device memory: the
    same values bit for bit, for a sorted state of two ragged species."""
    import torch

    p = inputs.config("c1_32", n_part=3001, n_species=2, m_ev=[0.05, 0.2], n_grid=16, n_steps=30, precision=prec,
                      seed=93)
    n = p["n_part"]
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(p["n_steps"])
        for s in range(2):
            pinned = [torch.empty(sh, dtype=torch.float64, pin_memory=True) for sh in ((3, n), (3, n), (n,))]
            pageable = [np.empty(sh) for sh in ((3, n), (3, n), (n,))]
            dev = [torch.empty(sh, dtype=torch.float64, device="cuda") for sh in ((3, n), (3, n), (n,))]
            F.fdf_get(r.ctx, s, *pinned)
            F.fdf_get(r.ctx, s, *pageable)
            F.fdf_get(r.ctx, s, *dev)
            for a, b, c in zip(pinned, pageable, dev):
                assert np.array_equal(a.numpy(), b) and np.array_equal(c.cpu().numpy(), b)
            # a NULL output next to page-locked ones
            xq = [torch.empty((3, n), dtype=torch.float64, pin_memory=True) for _ in range(2)]
            F.fdf_get(r.ctx, s, xq[0], xq[1], None)
            assert np.array_equal(xq[0].numpy(), pageable[0]) and np.array_equal(xq[1].numpy(), pageable[1])


@pytest.mark.parametrize("n_part", [1, 31, 33, 63, 65, 129])
def test_pass_chunk_edges(F, inputs, c1_tables, n_part):
    """Particle counts around the pass's work chunks (32 particles per warp, 64 in pairs):
    both launch shapes against the oracle, and equal to each other bit for bit."""
    p = inputs.config("c1_32", n_part=n_part, n_grid=8, n_steps=200, precision=1, seed=97)
    got = {}
    for pb in (2, 3):
        with F.Run(dict(p, pass_blocks=pb), c1_tables) as r:
            r.sample()
            r.step(p["n_steps"])
            got[pb] = r.get(0)
    for a, b in zip(got[2], got[3]):
        assert np.array_equal(a, b)
    ref = O.Oracle(p, c1_tables).run(np.arange(n_part))
    ex, eq, ew = errors(*got[2], ref, p["box"])
    assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)


# ---- inspection hooks --------------------------------------------------------------------------
@pytest.mark.parametrize("prec,n_steps,series", [(1, 200, 1), (1, 100, 0), (3, 100, 1), (0, 40, 0)])
def test_pass_info_reports_the_pass_kernel(F, inputs, c1_tables, prec, n_steps, series):
    """fdf_pass_info names the state form and whether every pass evaluated its step integrals
    as fitted polynomials or series: at 200 steps over the run the FP64-state form fits them
    (the throughput workloads' step size), at 100 it sums the nodes; the split-state form's
    drift series holds at 100 steps; the plain form always sums the nodes."""
    p = inputs.config("c1_32", n_part=2000, n_grid=16, n_steps=n_steps, precision=prec)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(n_steps)
        info = F.fdf_pass_info(r.ctx)
    print(prec, n_steps, info)
    assert info["form"] == {0: 0, 1: 1, 3: 2}[prec]
    assert info["series"] == series
    spp = 1 if prec == 0 else 4
    assert info["steps_per_pass"] == spp and info["passes"] == -(-n_steps // spp)


def test_pipe_rates_are_plausible(F):
    """The issue-rate probes behind the FP64 roofline: positive, and FP64 far below FP32."""
    d, f, c = F.fdf_pipe_rates()
    print("DFMA/s %.3e  FFMA/s %.3e  conversion round trips/s %.3e" % (d, f, c))
    assert d > 0 and f > 0 and c > 0
    assert f > 8 * d
