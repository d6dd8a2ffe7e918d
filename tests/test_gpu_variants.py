"""GPU parity of the paper's variants against the oracle.

* Interpolation order r = 2 (Sec. 4: the force read, the momentum transform
  and the deposit use the quadratic B-spline): whole runs in the plain FP64
  form (held to 1e-9) and in the split FP32 form (the contract's 1e-6 L,
  1e-5, 1e-5), two species of different masses, a ragged particle count.
* The delta-f momentum density (FDF_Q_W_QX..QZ), whose divergence gives the
  (1 + delta) theta spectrum of Sec. 4, against the oracle's deposit of the
  oracle's particles (relative L2 norm).
* The half-ensemble deposits (Sec. 4 takes power spectra as the cross-spectrum
  of two halves): even and odd ids against the oracle's deposit of those ids,
  and the two halves summing to the whole.
* The deposit's warp pre-sum (fdf_params.deposit_presum) against the oracle and
  against one atomic per particle and node.
* Super-steps (Sec. 2.1): the same schedule as the oracle's, one transform per
  super-step, and the run against the oracle's super-stepped run.
* The comparison equations of motion (Sec. 3.2 and 5) in the plain FP64 form.
* The exact eq:releq and eq:geodesic in the non-symplectic leapfrog (Sec. 3.3) in
  the plain FP64 form.
* The RMS of the four terms of eq:releq (Fig. 2) in every precision form.
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
    ex = np.max(np.abs(pdiff(x, ref["x"], L))) / L
    eq = np.max(np.linalg.norm(q - ref["q"], axis=0) / np.linalg.norm(ref["q"], axis=0))
    ew = np.max(np.abs(w - ref["w"]))
    return ex, eq, ew


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_tsc_runs_match_the_oracle(F, inputs, c1_tables, prec):
    p = inputs.config("c1_32", n_part=4099, n_species=2, m_ev=[0.05, 0.2], n_grid=32, n_steps=60, precision=prec,
                      seed=131, interp_order=2)
    o = O.Oracle(p, c1_tables)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(p["n_steps"])
        res = [r.get(s) for s in range(2)]
        dep = r.deposit(-1, F.FDF_Q_W_EPS)
    a = math.exp(o.lna(p["n_steps"]))
    dref = np.zeros_like(dep)
    for s in range(2):
        g = np.arange(s * p["n_part"], (s + 1) * p["n_part"])
        ref = o.run(g)
        ex, eq, ew = errors(*res[s], ref, p["box"])
        print("TSC prec %d species %d: x %.3e L, q %.3e, w %.3e" % (prec, s, ex, eq, ew))
        if prec == 0:
            assert ex < 1e-9 and eq < 1e-9 and ew < 1e-10, (ex, eq, ew)
        else:
            assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)
        dref += o.deposit(g, ref["x"], ref["q"], ref["w"], a, 0)
    err = np.linalg.norm(dep - dref) / np.linalg.norm(dref)
    print("TSC prec %d deposit: %.3e" % (prec, err))
    assert err < (1e-8 if prec == 0 else 1e-5)


@pytest.mark.parametrize("order", [1, 2])
def test_momentum_density_and_half_ensembles(F, inputs, c1_tables, order):
    p = inputs.config("c1_32", n_part=5000, n_grid=16, n_steps=30, precision=1, seed=137, interp_order=order)
    o = O.Oracle(p, c1_tables)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(p["n_steps"])
        mom = [r.deposit(-1, q) for q in (F.FDF_Q_W_QX, F.FDF_Q_W_QY, F.FDF_Q_W_QZ)]
        whole = r.deposit(-1, F.FDF_Q_W_EPS)
        halves = [r.deposit(-1, F.FDF_Q_W_EPS, parity) for parity in (0, 1)]
    g = np.arange(p["n_part"])
    ref = o.run(g)
    a = math.exp(o.lna(p["n_steps"]))
    for d, m in enumerate(mom):
        dref = o.deposit(g, ref["x"], ref["q"], ref["w"], a, 4 + d)
        err = np.linalg.norm(m - dref) / np.linalg.norm(dref)
        print("order %d momentum density %d: %.3e" % (order, d, err))
        assert err < 1e-5
    for parity, h in zip((0, 1), halves):
        sel = g[g % 2 == parity]
        dref = o.deposit(sel, ref["x"][:, sel], ref["q"][:, sel], ref["w"][sel], a, 0)
        err = np.linalg.norm(h - dref) / np.linalg.norm(dref)
        print("order %d half %d: %.3e" % (order, parity, err))
        assert err < 1e-5
    assert np.abs(halves[0] + halves[1] - whole).max() <= 1e-12 * np.abs(whole).max()


@pytest.mark.parametrize("prec,order", [(0, 1), (0, 2), (1, 1), (1, 2), (3, 1)])
def test_deposit_presum_matches_the_oracle(F, inputs, c1_tables, prec, order):
    """The deposit with the warp pre-sum (fdf_params.deposit_presum = 1) against the
    oracle's deposit and against one atomic per particle and node.  About ten
    particles per cell and two ragged species, so that a warp's sets of particles
    sharing a base cell run from one lane to many (every level of the shuffle tree)
    and the last warp of each species is partly empty; the half-ensemble deposits
    leave every other lane out of the sums."""
    p = inputs.config("c1_32", n_part=5003, n_species=2, m_ev=[0.05, 0.2], n_grid=8, n_steps=20, precision=prec,
                      seed=139, interp_order=order)
    o = O.Oracle(p, c1_tables)
    got = {}
    for presum in (1, -1):
        with F.Run(dict(p, deposit_presum=presum), c1_tables) as r:
            r.sample()
            r.step(p["n_steps"])
            got[presum] = [r.deposit(-1, F.FDF_Q_W_EPS)] + [r.deposit(-1, F.FDF_Q_W_EPS, par) for par in (0, 1)] + \
                          [r.deposit(-1, F.FDF_Q_W_QX)]
    a = math.exp(o.lna(p["n_steps"]))
    refs = [np.zeros((8, 8, 8)) for _ in range(4)]
    for s in range(2):
        g = np.arange(s * p["n_part"], (s + 1) * p["n_part"])
        ref = o.run(g)
        refs[0] += o.deposit(g, ref["x"], ref["q"], ref["w"], a, 0)
        for par in (0, 1):
            sel = (g % 2) == par
            refs[1 + par] += o.deposit(g[sel], ref["x"][:, sel], ref["q"][:, sel], ref["w"][sel], a, 0)
        refs[3] += o.deposit(g, ref["x"], ref["q"], ref["w"], a, 4)
    bar = 1e-8 if prec == 0 else 1e-5
    for k, (dep, dref) in enumerate(zip(got[1], refs)):
        err = np.linalg.norm(dep - dref) / np.linalg.norm(dref)
        same = np.abs(dep - got[-1][k]).max() / np.abs(got[-1][k]).max()
        print("prec %d order %d deposit %d: against the oracle %.3e, against the plain deposit %.3e"
              % (prec, order, k, err, same))
        assert err < bar
        assert same <= 1e-12


def test_bad_deposit_arguments_are_refused(F, inputs, c1_tables):
    p = inputs.config("c1_32", n_part=100, n_grid=8, n_steps=2, precision=1)
    with F.Run(p, c1_tables) as r:
        r.sample()
        for quantity, parity in ((7, -1), (-1, -1), (0, 2), (0, -2)):
            with pytest.raises(F.FdfError) as e:
                r.deposit(-1, quantity, parity)
            assert e.value.code == F.FDF_EINVAL
    with pytest.raises(F.FdfError):
        F.fdf_footprint(F.make_params(dict(p, interp_order=3)))


# ---- super-steps (Sec. 2.1) ------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1, 3])
def test_supersteps_match_the_oracle(F, inputs, c1_tables, prec):
    """The library's schedule equals the oracle's; each super-step is built by transform
    once per run (the y pass counts the transforms); the run matches the oracle's
    super-stepped run at the usual bars."""
    p = inputs.config("c1_32", n_part=3000, n_grid=16, n_steps=80, precision=prec, seed=141, superstep_tol=0.01)
    o = O.Oracle(p, c1_tables)
    want = o.supersteps()
    assert 2 < want.sum() < p["n_steps"] // 2, want.sum()
    with F.Run(p, c1_tables) as r:
        got = r.supersteps()
        assert np.array_equal(got, want), (np.flatnonzero(got), np.flatnonzero(want))
        F.fdf_timing(r.ctx, True)
        r.sample()
        r.step(p["n_steps"])
        builds = F.fdf_kernel_time(r.ctx, F.FDF_K_FIELDS_Y)[1]
        F.fdf_timing(r.ctx, False)
        res = r.get(0)
    print("super-steps: %d of %d steps built by transform (%d builds)" % (want.sum(), p["n_steps"] + 1, builds))
    assert builds == want.sum()
    ref = o.run(np.arange(p["n_part"]))
    ex, eq, ew = errors(*res, ref, p["box"])
    print("super-steps prec %d: x %.3e L, q %.3e, w %.3e" % (prec, ex, eq, ew))
    if prec == 0:
        assert ex < 1e-9 and eq < 1e-9 and ew < 1e-10, (ex, eq, ew)
    else:
        assert ex < TOL_X and eq < TOL_Q and ew < TOL_W, (ex, eq, ew)
    # and the super-steps do change the result (the fields are interpolated)
    exact = O.Oracle(dict(p, superstep_tol=0.0), c1_tables).run(np.arange(p["n_part"]))
    assert np.max(np.abs(exact["q"] - ref["q"])) > 0


def test_superstep_schedule_of_the_throughput_workload(F, inputs):
    p = inputs.config("c3_3x256", n_part=1000, superstep_tol=0.01)
    tables = inputs.transfer_tables(p)
    with F.Run(p, tables) as r:
        got = r.supersteps()
    want = O.Oracle(p, tables).supersteps()
    print("3 x 256^3 workload: %d of %d steps built by transform" % (want.sum(), p["n_steps"] + 1))
    assert np.array_equal(got, want)


# ---- equations of motion (Sec. 3.2, 3.3, 5) ---------------------------------------------------
@pytest.mark.parametrize("eom", [1, 2, 3, 4])
def test_comparison_equations_of_motion_match_the_oracle(F, inputs, c1_tables, eom):
    """The comparison forms of the kick (canonical P, special-relativistic with Newtonian
    gravity, the simpler q form, Newtonian acceleration) in the plain FP64 form against
    the oracle, and each differs from the method's own form."""
    p = inputs.config("c1_32", n_part=2000, n_species=2, m_ev=[0.05, 0.2], n_grid=16, n_steps=40, precision=0,
                      seed=151, eom=eom)
    o = O.Oracle(p, c1_tables)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(p["n_steps"])
        res = [r.get(s) for s in range(2)]
    for s in range(2):
        g = np.arange(s * p["n_part"], (s + 1) * p["n_part"])
        ref = o.run(g)
        ex, eq, ew = errors(*res[s], ref, p["box"])
        print("eom %d species %d: x %.3e L, q %.3e, w %.3e" % (eom, s, ex, eq, ew))
        assert ex < 1e-9 and eq < 1e-9 and ew < 1e-10, (ex, eq, ew)
    base = O.Oracle(dict(p, eom=0), c1_tables).run(np.arange(p["n_part"]))
    assert np.max(np.abs(base["q"] - res[0][1])) > 1e-3 * np.max(np.abs(base["q"] - base["qs"]))


# ---- the exact equations of motion, non-symplectic (Sec. 3.3) ----------------------------------
@pytest.mark.parametrize("spp,order,ss", [(1, 1, 0.0), (2, 2, 0.0), (2, 1, 0.01)])
def test_exact_equations_of_motion_match_the_oracle(F, inputs, c1_tables, spp, order, ss):
    """FDF_EOM_EXACT (eq:releq and eq:geodesic in the non-symplectic leapfrog) in the
    plain FP64 form against the oracle: two species, one and two steps per pass, CIC and
    TSC, with super-steps (the phi + psi grids are interpolated too), the run split in
    two calls; and it differs from the method's separable form."""
    p = inputs.config("c1_32", n_part=3001, n_species=2, m_ev=[0.05, 0.2], n_grid=16, n_steps=40, precision=0,
                      seed=161, eom=F.FDF_EOM_EXACT, steps_per_pass=spp, interp_order=order, superstep_tol=ss)
    o = O.Oracle(p, c1_tables)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(17)
        r.step(p["n_steps"] - 17)
        res = [r.get(s) for s in range(2)]
    for s in range(2):
        g = np.arange(s * p["n_part"], (s + 1) * p["n_part"])
        ref = o.run(g)
        ex, eq, ew = errors(*res[s], ref, p["box"])
        print("exact eom, %d steps per pass, order %d, super-steps %g, species %d: x %.3e L, q %.3e, w %.3e"
              % (spp, order, ss, s, ex, eq, ew))
        assert ex < 1e-9 and eq < 1e-9 and ew < 1e-10, (ex, eq, ew)
    base = O.Oracle(dict(p, eom=0), c1_tables).run(np.arange(p["n_part"]))
    d = np.max(np.linalg.norm(base["q"] - res[0][1], axis=0) / np.linalg.norm(base["q"], axis=0))
    print("exact against the separable form: largest |dq| / |q| %.3e" % d)
    assert d > 1e-9


# ---- the four terms of eq:releq (Fig. 2) --------------------------------------------------------
@pytest.mark.parametrize("prec,order", [(0, 1), (1, 1), (1, 2), (2, 1), (3, 1)])
def test_accel_terms_match_the_oracle(F, inputs, c1_tables, prec, order):
    """fdf_accel_terms against the oracle's on the oracle's own particles, per species and
    for all, at an early step (relativistic: the first two terms alike) and a late one.
    Every term, the q phi_dot term included, is held to one bar per precision: the steps'
    grids transform phi_dot alone (its packed partner, slot 7, is zero there), so its FP32
    rounding is relative to phi_dot itself."""
    p = inputs.config("c1_32", n_part=3001, n_species=2, m_ev=[0.05, 0.2], n_grid=16, n_steps=60, precision=prec,
                      seed=181, interp_order=order)
    o = O.Oracle(p, c1_tables)
    tol = {0: 1e-9, 1: 1e-6, 2: 3e-3, 3: 1e-6}[prec]
    tol_dot = tol
    with F.Run(p, c1_tables) as r:
        r.sample()
        done = 0
        for k in (5, 60):
            r.step(k - done)
            done = k
            got = [r.accel_terms(s) for s in (0, 1, -1)]
            ref = []
            for s in range(2):
                g = np.arange(s * p["n_part"], (s + 1) * p["n_part"])
                st = o.run(g, k_to=k)
                ref.append(o.accel_terms(g, st["x"], st["q"], k))
            g = np.arange(2 * p["n_part"])
            st = o.run(g, k_to=k)
            ref.append(o.accel_terms(g, st["x"], st["q"], k))
            for s, gv, rv in zip((0, 1, -1), got, ref):
                rel = np.abs(gv - rv) / rv
                print("prec %d order %d step %d species %2d: rms %s  (rel. err %.2e, phi_dot term %.2e)"
                      % (prec, order, k, s, " ".join("%.3e" % v for v in gv), np.delete(rel, 3).max(), rel[3]))
                assert np.delete(rel, 3).max() < tol and rel[3] < tol_dot, (s, gv, rv)
