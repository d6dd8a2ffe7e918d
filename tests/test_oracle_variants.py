"""Pins of the oracle's paper variants.

* Interpolation order r = 2 (Sec. 4 offers r = 1 and r = 2), the quadratic
  B-spline (triangular-shaped cloud) on the node grid:
  - its weights at a node are 3/4 and 1/8, 1/8 per axis (a unit spike at node j
    read at node j gives (3/4)^3, at a face neighbour (3/4)^2 (1/8), ...);
  - it reproduces constants and linear fields exactly (the first moment of a
    centred B-spline is preserved);
  - the deposit is the transpose of the gather: sum_n grid_n F_n =
    sum_k v_k F(x_k) for any field F (checked for both orders), and conserves
    the deposited total.
* Super-steps (Sec. 2.1): the schedule rule, the change measure in closed form,
  and exactness for fields linear in ln a.
* The equations of motion (eq:releq_approx, eq:releq_lag, eq:p_eq, eq:q_eq and
  the Newtonian acceleration): the total kick under uniform fields in closed form.
* The exact eq:releq and eq:geodesic in the non-symplectic leapfrog (eom 5, the
  check of Sec. 3.3): convergence to scipy's ODE solution of those equations,
  the (1 + phi + psi) drift scaling, no force on a momentum parallel to grad phi,
  and the phi + psi slot against the spectral gradient of grad phi.
* The delta-f momentum density (quantities 4-6: w q_x, w q_y, w q_z), the
  moment whose divergence gives the (1 + delta) theta spectrum of Sec. 4: it
  is the deposit of v = w q_d, checked through the transpose identity against
  an independent sum.
"""
import math

import numpy as np
import pytest

import oracle as O


def _oracle(inputs, c1_tables, order):
    p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=40, seed=21, interp_order=order)
    return O.Oracle(p, c1_tables), p


def test_tsc_weights_at_nodes(inputs, c1_tables):
    o, p = _oracle(inputs, c1_tables, 2)
    N, L = p["n_grid"], p["box"]
    h = L / N
    F = np.zeros((8, N, N, N))
    F[:, 7, 5, 3] = 1.0            # spike at node (x=3, y=5, z=7)
    at = lambda ix, iy, iz: o.gather(F, [ix * h, iy * h, iz * h])[0]
    assert at(3, 5, 7) == pytest.approx(0.75 ** 3, abs=1e-15)
    assert at(4, 5, 7) == pytest.approx(0.75 ** 2 * 0.125, abs=1e-15)
    assert at(4, 6, 7) == pytest.approx(0.75 * 0.125 ** 2, abs=1e-15)
    assert at(2, 4, 6) == pytest.approx(0.125 ** 3, abs=1e-15)
    assert at(5, 5, 7) == 0.0
    # periodic neighbour across the box edge
    F[:] = 0.0
    F[:, 0, 0, 0] = 1.0
    assert o.gather(F, [(N - 1) * h, 0.0, 0.0])[0] == pytest.approx(0.75 ** 2 * 0.125, abs=1e-15)


def test_tsc_reproduces_constants_and_linear_fields(inputs, c1_tables):
    o, p = _oracle(inputs, c1_tables, 2)
    N, L = p["n_grid"], p["box"]
    h = L / N
    rng = np.random.default_rng(8)
    const = np.full((8, N, N, N), 2.5)
    n = np.arange(N, dtype=float)
    z, y, x = np.meshgrid(n, n, n, indexing="ij")
    lin = np.stack([x - 3 * y + 7 * z] * 8)
    for _ in range(50):
        u = rng.uniform(1.5, N - 2.5, 3)     # the 3-node stencil stays clear of the wrap
        assert np.allclose(o.gather(const, u * h), 2.5, rtol=0, atol=1e-14)
        assert np.allclose(o.gather(lin, u * h), u[0] - 3 * u[1] + 7 * u[2], rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_is_the_transpose_of_the_gather(inputs, c1_tables, order):
    o, p = _oracle(inputs, c1_tables, order)
    N, L = p["n_grid"], p["box"]
    rng = np.random.default_rng(11 + order)
    n = 500
    x = rng.uniform(0, L, (3, n))
    q = rng.standard_normal((3, n)) * 5e-4
    w = rng.standard_normal(n) * 1e-3
    F = rng.standard_normal((8, N, N, N))
    reads = np.array([o.gather(F, x[:, k])[0] for k in range(n)])
    a = 1 / 32
    grid = o.deposit(np.zeros(n, np.int64), x, q, w, a, 1)
    assert abs((grid * F[0]).sum() - (w * reads).sum()) < 1e-12 * np.abs(w * reads).sum()
    assert abs(grid.sum() - w.sum()) < 1e-13 * np.abs(w).sum()
    # the momentum density, component by component
    for d in range(3):
        gq = o.deposit(np.zeros(n, np.int64), x, q, w, a, 4 + d)
        v = w * q[d]
        assert abs((gq * F[0]).sum() - (v * reads).sum()) < 1e-12 * np.abs(v * reads).sum()


def test_tsc_deposit_of_a_particle_on_a_node(inputs, c1_tables):
    o, p = _oracle(inputs, c1_tables, 2)
    N, L = p["n_grid"], p["box"]
    h = L / N
    x = np.array([[3 * h], [5 * h], [7 * h]])
    q = np.full((3, 1), 1e-4)
    g = o.deposit(np.zeros(1, np.int64), x, q, np.array([2.0]), 1 / 32, 1)
    assert g[7, 5, 3] == pytest.approx(2 * 0.75 ** 3, abs=1e-15)
    assert g[8, 6, 4] == pytest.approx(2 * 0.125 ** 3, abs=1e-15)
    assert np.count_nonzero(g) == 27


# ---- super-steps (Sec. 2.1) ------------------------------------------------------------------
def _ss_oracle(inputs, tables, tol, **over):
    p = inputs.config("c1_32", n_grid=8, n_part=300, n_steps=40, seed=23, superstep_tol=tol)
    p.update(over)
    return O.Oracle(p, tables), p


def test_superstep_schedule_rule(inputs, c1_tables):
    """Every step inside an interval changes the tables by at most tol from its
    first super-step; each super-step after the first exceeds tol from the one
    before; the ends are super-steps; tol = 0 computes every step."""
    o, p = _ss_oracle(inputs, c1_tables, 0.01)
    s = o.supersteps()
    n = p["n_steps"]
    assert s[0] == 1 and s[n] == 1
    sup = np.flatnonzero(s)
    assert 2 < len(sup) < n + 1
    for a, b in zip(sup[:-1], sup[1:]):
        for k in range(a + 1, b):
            assert o.tf_change(a, k) <= 0.01
        if b != n:
            assert o.tf_change(a, b) > 0.01
    o0, _ = _ss_oracle(inputs, c1_tables, 0.0)
    assert np.all(o0.supersteps() == 1)


def test_superstep_change_closed_form(inputs, c1_tables):
    """Tables T = c(k) (1 + b ln a): the change between two steps is |b| |ln a1 - ln a0| / |1 + b ln a0| scaled by
    the same c, so it has a closed form, and tables constant in a never trigger a super-step."""
    t = {k: np.array(v, copy=True) for k, v in c1_tables.items()}
    lna = t["lna"]
    b = 0.01
    ck = 1.0 + 0.5 * np.cos(t["lnk"])
    for key in ("T_psi", "T_phi"):
        t[key] = ck[None, :] * (1.0 + b * lna[:, None])
    o, p = _ss_oracle(inputs, t, 0.01)
    for j0, j1 in ((0, 5), (10, 30), (3, 4)):
        l0, l1 = o.lna(j0), o.lna(j1)
        want = abs(b * (l1 - l0)) / abs(1.0 + b * l0)
        assert o.tf_change(j0, j1) == pytest.approx(want, rel=1e-9)
    for key in ("T_psi", "T_phi"):
        t[key] = np.tile(ck, (len(lna), 1))
    oc, pc = _ss_oracle(inputs, t, 0.01)
    s = oc.supersteps()
    assert s.sum() == 2 and s[0] == 1 and s[-1] == 1


def test_supersteps_exact_for_tables_linear_in_ln_a(inputs, c1_tables):
    """Fields that are linear in ln a are reproduced exactly by the interpolation, so a
    super-stepped run equals the run that computes every step (to rounding); a
    plausible slip (interpolating in a, or weighting the wrong end) breaks it."""
    t = {k: np.array(v, copy=True) for k, v in c1_tables.items()}
    lna = t["lna"]
    ck = 1e-5 * (1.0 + np.sin(t["lnk"]))
    # psi linear in ln a; phi constant, so phi_dot = a H dT_phi/d ln a = 0 (a H itself is
    # not linear in ln a and would not interpolate exactly)
    t["T_psi"] = ck[None, :] * (2.0 + 0.05 * lna[:, None])
    t["T_phi"] = np.tile(1.5 * ck, (len(lna), 1))
    t["dTphi_dlna"] = np.zeros_like(t["T_phi"])
    o, p = _ss_oracle(inputs, t, 0.05)
    assert 2 < o.supersteps().sum() < p["n_steps"] // 2
    o0, _ = _ss_oracle(inputs, t, 0.0)
    g = np.arange(p["n_part"])
    a, b = o.run(g), o0.run(g)
    assert np.max(np.abs(a["x"] - b["x"])) < 1e-9 * p["box"]
    assert np.max(np.abs(a["q"] - b["q"]) / np.abs(b["q"]).max()) < 1e-12
    # with the synthetic tables (not linear in ln a) the runs differ, but only a little
    o1, _ = _ss_oracle(inputs, c1_tables, 0.01)
    o2, _ = _ss_oracle(inputs, c1_tables, 0.0)
    r1, r2 = o1.run(g), o2.run(g)
    dq = np.max(np.linalg.norm(r1["q"] - r2["q"], axis=0) / np.linalg.norm(r2["q"], axis=0))
    assert 0 < dq < 1e-3


# ---- equations of motion (Sec. 3.2, 3.3, 5) ---------------------------------------------------
def _quad(o, f, l0, l1, n=200):
    from scipy import integrate
    edges = np.linspace(l0, l1, n + 1)
    return math.fsum(integrate.quad(lambda s: f(math.exp(s)) / (math.exp(s) * o.hubble(math.exp(s))), a, b,
                                    epsrel=1e-13, epsabs=0)[0] for a, b in zip(edges[:-1], edges[1:]))


@pytest.mark.parametrize("eom", [0, 1, 2, 3, 4])
def test_eom_kicks_under_uniform_fields(inputs, c1_tables, eom):
    """With frozen uniform fields every variant's total kick over a run is a closed form
    in integrals over conformal time (scipy quadrature here):
      0: -grad psi int eps0 - (q0^2 grad phi - q0 (q0.grad phi)) int 1/eps0 + q0 phi_dot int 1
      1: -grad psi int eps0 - q0^2 grad phi int 1/eps0
      2: -grad psi int (2 q0^2 + m^2 a^2)/eps0
      3: -grad psi int eps0
      4: -grad psi m int a
    with eps0 = sqrt(q0^2 + m^2 a^2).  A dropped or swapped term changes the result
    by far more than the quadrature error."""
    m = 0.05
    p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=30, seed=21, m_ev=[m], eom=eom)
    N = p["n_grid"]
    gpsi, gphi, cdot = np.array([2e-6, -1e-6, 5e-7]), np.array([-3e-7, 4e-7, 1e-6]), 3e-9
    frozen = inputs.uniform_fields(N, gpsi, gphi, cdot, 0.0)
    o = O.Oracle(p, c1_tables)
    g = np.arange(8)
    ic = o.initial(g, frozen=np.zeros_like(frozen))
    x, q = o.integrate(g, ic["x"], ic["q"], ic["q0"], 0, p["n_steps"], frozen=frozen)
    l0, l1 = o.lna(0), o.lna(p["n_steps"])
    for i in range(len(g)):
        q0 = ic["q0"][:, i]
        q02 = q0 @ q0
        e = lambda a: math.sqrt(q02 + m * m * a * a)
        if eom == 0:
            dq = (-gpsi * _quad(o, e, l0, l1) - (q02 * gphi - q0 * (q0 @ gphi)) * _quad(o, lambda a: 1 / e(a), l0, l1)
                  + q0 * cdot * _quad(o, lambda a: 1.0, l0, l1))
        elif eom == 1:
            dq = -gpsi * _quad(o, e, l0, l1) - q02 * gphi * _quad(o, lambda a: 1 / e(a), l0, l1)
        elif eom == 2:
            dq = -gpsi * _quad(o, lambda a: (2 * q02 + m * m * a * a) / e(a), l0, l1)
        elif eom == 3:
            dq = -gpsi * _quad(o, e, l0, l1)
        else:
            dq = -gpsi * m * _quad(o, lambda a: a, l0, l1)
        assert np.linalg.norm(q[:, i] - q0 - dq) < 1e-10 * np.linalg.norm(dq), (eom, i)


# ---- the exact equations of motion in the non-symplectic leapfrog (Sec. 3.3) ---------------
def _exact_ode_solution(o, m, x0, q0, l0, l1, gpsi, gphi, cdot, s):
    """eq:releq and eq:geodesic under uniform fields, integrated in ln a by scipy's DOP853."""
    from scipy.integrate import solve_ivp

    def f(l, y):
        a = math.exp(l)
        q = y[3:]
        e = math.sqrt(q @ q + m * m * a * a)
        dx = q / e * (1.0 + s)
        dq = -e * gpsi - (q @ q) / e * gphi + q * (q @ gphi) / e + q * cdot
        return np.concatenate([dx, dq]) / (a * o.hubble(a))

    sol = solve_ivp(f, (l0, l1), np.concatenate([x0, q0]), method="DOP853", rtol=1e-12, atol=1e-14)
    assert sol.success
    return sol.y[:3, -1], sol.y[3:, -1]


def test_exact_eom_converges_to_the_ode_solution(inputs, c1_tables):
    """eom 5 integrates eq:releq and eq:geodesic themselves, so under uniform fields its
    leapfrog converges to an ODE solver's solution of those equations as the step shrinks
    (first order in q: each half kick holds q at its start), while the method's separable
    form (eom 0) converges to a different curve."""
    m = 0.05
    gpsi, gphi, cdot, s = np.array([2e-6, -1e-6, 5e-7]), np.array([-3e-7, 4e-7, 1e-6]), 3e-9, 1e-3
    g = np.arange(4)
    err = {}
    for ns in (60, 240):
        p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=ns, seed=21, m_ev=[m], eom=5)
        L = p["box"]
        frozen = inputs.uniform_fields(p["n_grid"], gpsi, gphi, cdot, s)
        o = O.Oracle(p, c1_tables)
        ic = o.initial(g, frozen=np.zeros_like(frozen))
        x, q = o.integrate(g, ic["x"], ic["q"], ic["q0"], 0, ns, frozen=frozen)
        xs, qs = O.Oracle(dict(p, eom=0), c1_tables).integrate(g, ic["x"], ic["q"], ic["q0"], 0, ns, frozen=frozen)
        ex = eq = eq_sep = 0.0
        for i in range(len(g)):
            xe, qe = _exact_ode_solution(o, m, ic["x"][:, i], ic["q"][:, i], o.lna(0), o.lna(ns), gpsi, gphi, cdot, s)
            moved = np.linalg.norm((xe - ic["x"][:, i] + L / 2) % L - L / 2)
            kicked = np.linalg.norm(qe - ic["q"][:, i])
            ex = max(ex, np.linalg.norm((x[:, i] - xe + L / 2) % L - L / 2) / moved)
            eq = max(eq, np.linalg.norm(q[:, i] - qe) / kicked)
            eq_sep = max(eq_sep, np.linalg.norm(qs[:, i] - qe) / kicked)
        err[ns] = (ex, eq, eq_sep)
        print("exact eom, %d steps: x %.2e of the displacement, q %.2e of the kick (separable form: %.2e)"
              % (ns, ex, eq, eq_sep))
    assert err[240][0] < 1e-5 and err[240][1] < 3e-5
    assert err[240][1] < err[60][1] / 3          # first order in the step
    assert err[240][2] > 30 * err[240][1]         # eom 0 is another equation


def test_exact_eom_invariants(inputs, c1_tables):
    """Two exact properties of eq:releq and eq:geodesic that a sign or factor slip breaks:
    * with no gradients and no phi_dot, q is constant and the drift is (1 + phi + psi)
      times the drift with phi + psi = 0;
    * with grad psi = 0 and phi_dot = 0, a momentum parallel to grad phi feels no force
      (-(q^2/eps) grad phi + q (q.grad phi)/eps vanishes), so it never changes."""
    # a box much larger than the distance travelled, so that no wrap hides the scaling
    p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=40, seed=21, m_ev=[0.05], eom=5, box=1e5)
    L, N = p["box"], p["n_grid"]
    o = O.Oracle(p, c1_tables)
    g = np.arange(6)
    ic = o.initial(g, frozen=np.zeros((8, N, N, N)))
    x0 = np.full((3, len(g)), L / 2)
    s = 2e-3
    xa, qa = o.integrate(g, x0, ic["q"], ic["q0"], 0, p["n_steps"],
                         frozen=inputs.uniform_fields(N, np.zeros(3), np.zeros(3), 0.0, s))
    xb, qb = o.integrate(g, x0, ic["q"], ic["q0"], 0, p["n_steps"],
                         frozen=inputs.uniform_fields(N, np.zeros(3), np.zeros(3), 0.0, 0.0))
    assert np.array_equal(qa, ic["q"]) and np.array_equal(qb, ic["q"])
    da, db = (xa - x0 + L / 2) % L - L / 2, (xb - x0 + L / 2) % L - L / 2
    assert np.max(np.abs(da - (1 + s) * db)) <= 1e-12 * np.max(np.abs(da))
    gphi = np.array([3e-6, -2e-6, 1e-6])
    qpar = np.outer(gphi / np.linalg.norm(gphi), np.linalg.norm(ic["q"], axis=0))
    _, qc = o.integrate(g, x0, qpar, qpar, 0, p["n_steps"],
                        frozen=inputs.uniform_fields(N, np.zeros(3), gphi, 0.0, 0.0))
    assert np.max(np.linalg.norm(qc - qpar, axis=0) / np.linalg.norm(qpar, axis=0)) < 1e-14
    # the method's separable form does feel it (q0 is parallel too, so it also vanishes there):
    # break the parallelism and the force appears
    qtilt = qpar + 0.3 * np.roll(qpar, 1, axis=0)
    _, qd = o.integrate(g, x0, qtilt, qtilt, 0, p["n_steps"],
                        frozen=inputs.uniform_fields(N, np.zeros(3), gphi, 0.0, 0.0))
    assert np.min(np.linalg.norm(qd - qtilt, axis=0) / np.linalg.norm(qtilt, axis=0)) > 1e-6


def test_phi_plus_psi_slot_is_psi_plus_the_potential_of_grad_phi(inputs, c1_tables):
    """The exact drift reads phi + psi from slot 7 built with OR_SLOT7_PHI_PLUS_PSI.  Its
    difference from the plain slot 7 (psi) is phi, whose spectral gradient must equal the
    grad phi slots 3-5, which are built from the same transfer function independently."""
    p = inputs.config("c1_32", n_grid=16, seed=23)
    o = O.Oracle(p, c1_tables)
    R = o.noise()
    lna = o.lna(60)
    plain, _ = o.fields(lna, 0xFF, R)
    summed, _ = o.fields(lna, 0xFF | 0x100, R)
    assert np.array_equal(plain[:7], summed[:7])
    phi = summed[7] - plain[7]
    N, kf = p["n_grid"], 2 * math.pi / p["box"]
    n = np.fft.fftfreq(N, 1.0 / N)
    Phi = np.fft.fftn(phi)
    for d, axis in ((0, 2), (1, 1), (2, 0)):          # layout [z][y][x]
        shape = [1, 1, 1]
        shape[axis] = N
        grad = np.fft.ifftn(1j * kf * n.reshape(shape) * Phi).real
        ref = plain[3 + d]
        assert np.max(np.abs(grad - ref)) < 1e-10 * np.max(np.abs(ref)), d
    assert np.max(np.abs(phi)) > 0.1 * np.max(np.abs(plain[7]))


# ---- the four terms of eq:releq (Fig. 2) ------------------------------------------------------
def test_accel_terms_exact_cases(inputs, c1_tables):
    """Closed cases of the RMS of -eps grad psi, -(q^2/eps) grad phi, q (q.grad phi)/eps,
    q phi_dot and of their sum, under uniform fields:
    * a momentum parallel to grad phi: the two grad phi terms cancel (the sum has only
      the grad psi term), a perpendicular one: the third term vanishes;
    * massless particles (eps = |q|): the first two terms are |q| |grad psi| and
      |q| |grad phi|;
    * phi_dot alone: the fourth term is |phi_dot| |q|, the others vanish."""
    p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=40, seed=21, m_ev=[0.05])
    N = p["n_grid"]
    o = O.Oracle(p, c1_tables)
    g = np.arange(64)
    ic = o.initial(g, frozen=np.zeros((8, N, N, N)))
    x = ic["x"]
    qn = np.linalg.norm(ic["q"], axis=0)
    k = 25
    a = math.exp(o.lna(k))
    m = p["m_ev"][0]
    eps = np.sqrt(qn ** 2 + (m * a) ** 2)
    gpsi, gphi = np.array([2e-6, -1e-6, 5e-7]), np.array([-3e-7, 4e-7, 1e-6])
    # parallel to grad phi
    qpar = np.outer(gphi / np.linalg.norm(gphi), qn)
    r = o.accel_terms(g, x, qpar, k, frozen=inputs.uniform_fields(N, gpsi, gphi, 0.0, 0.0))
    assert abs(r[1] - r[2]) <= 1e-14 * r[1] and r[1] > 0
    assert abs(r[4] - r[0]) <= 1e-14 * r[0]
    assert math.isclose(r[0], np.linalg.norm(gpsi) * math.sqrt(np.mean(eps ** 2)), rel_tol=1e-13)
    # perpendicular to grad phi
    perp = np.cross(gphi, [1.0, 0.0, 0.0])
    qperp = np.outer(perp / np.linalg.norm(perp), qn)
    r = o.accel_terms(g, x, qperp, k, frozen=inputs.uniform_fields(N, np.zeros(3), gphi, 0.0, 0.0))
    assert r[2] <= 1e-14 * r[1] and r[0] == 0.0 and r[3] == 0.0
    assert math.isclose(r[1], np.linalg.norm(gphi) * math.sqrt(np.mean((qn ** 2 / eps) ** 2)), rel_tol=1e-13)
    assert abs(r[4] - r[1]) <= 1e-14 * r[1]
    # massless
    o0 = O.Oracle(dict(p, m_ev=[0.0]), c1_tables)
    r = o0.accel_terms(g, x, ic["q"], k, frozen=inputs.uniform_fields(N, gpsi, gphi, 0.0, 0.0))
    rq = math.sqrt(np.mean(qn ** 2))
    assert math.isclose(r[0], np.linalg.norm(gpsi) * rq, rel_tol=1e-13)
    assert math.isclose(r[1], np.linalg.norm(gphi) * rq, rel_tol=1e-13)
    # phi_dot alone
    r = o.accel_terms(g, x, ic["q"], k, frozen=inputs.uniform_fields(N, np.zeros(3), np.zeros(3), 3e-9, 0.0))
    assert r[0] == r[1] == r[2] == 0.0
    assert math.isclose(r[3], 3e-9 * math.sqrt(np.mean(qn ** 2)), rel_tol=1e-13) and r[4] == r[3]


def test_accel_terms_follow_the_paper_trend(inputs, c1_tables):
    """Fig. 2's reading of eq:releq on a run with built fields: the Newtonian term's share
    grows as the particles become non-relativistic (eps/|q| grows with a), while the two
    quadratic terms stay of one order."""
    p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=60, seed=29, m_ev=[0.1])
    o = O.Oracle(p, c1_tables)
    g = np.arange(2000)
    ic = o.initial(g)
    x, q = ic["x"], ic["q"]
    ratios = []
    for k0, k1 in ((0, 5), (5, 60)):
        x, q = o.integrate(g, x, q, ic["q0"], k0, k1)
        r = o.accel_terms(g, x, q, k1)
        print("step %d: rms terms %s" % (k1, " ".join("%.3e" % v for v in r)))
        assert 0.05 < r[2] / r[1] < 2.0
        ratios.append(r[0] / r[1])
    assert ratios[1] > 3 * ratios[0]
