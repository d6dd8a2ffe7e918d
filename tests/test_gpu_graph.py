"""fdf_run_graph: a whole run (fdf_sample + fdf_step(n)) recorded once as a CUDA
graph and replayed.

The replay must be the run: every particle's position, momentum and weight
bitwise equal to the sequential calls' (each particle's arithmetic is the same),
the deposit equal up to the order of its FP64 atomic additions, the launch count
the same, and the context left where the sequential calls leave it, so that
fdf_step can carry on from there.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


def _results(F, r, p):
    parts = [r.get(s) for s in range(p["n_species"])]
    return parts, r.deposit(-1, F.FDF_Q_W_EPS)


def _same(a, b):
    (pa, da), (pb, db) = a, b
    for (x, q, w), (x0, q0, w0) in zip(pa, pb):
        assert np.array_equal(x, x0) and np.array_equal(q, q0) and np.array_equal(w, w0)
    assert np.max(np.abs(da - db)) <= 1e-12 * np.max(np.abs(db))


CASES = [dict(precision=1), dict(precision=1, superstep_tol=0.01), dict(precision=2), dict(precision=3),
         dict(precision=4), dict(precision=0), dict(precision=0, eom=5)]


@pytest.mark.parametrize("over", CASES, ids=["f32", "f32-supersteps", "bf16", "f32-fixed", "bf16-fixed", "f64",
                                             "f64-exact"])
def test_replay_equals_the_sequential_run(F, inputs, c1_tables, over):
    p = inputs.config("c1_32", n_part=9001, n_species=2, m_ev=[0.05, 0.2], n_grid=32, n_steps=37, seed=171,
                      **over)
    n = p["n_steps"]
    with F.Run(p, c1_tables) as r:
        l0 = F.fdf_launch_count(r.ctx)
        r.sample()
        r.step(n)
        launches = F.fdf_launch_count(r.ctx) - l0
        ref = _results(F, r, p)
    with F.Run(p, c1_tables) as r:
        for rep in range(3):                  # the recording run, then two replays
            l0 = F.fdf_launch_count(r.ctx)
            r.run_graph(n)
            assert F.fdf_launch_count(r.ctx) - l0 == launches
            assert r.state()[0] == n
            _same(_results(F, r, p), ref)
    print("%s: %d launches per run, replays bitwise equal" % (over, launches))


def test_replay_then_steps_equals_the_sequential_calls(F, inputs, c1_tables):
    """After a replay of 20 steps the context carries on with fdf_step (sorts, buffers
    and the step counter as the sequential calls left them); a run of another length
    records a new graph; sequential runs still work on the same context."""
    p = inputs.config("c1_32", n_part=9001, n_species=2, m_ev=[0.05, 0.2], n_grid=32, n_steps=37, seed=173,
                      precision=1)
    with F.Run(p, c1_tables) as r:
        r.sample()
        r.step(20)
        r.step(17)
        ref37 = _results(F, r, p)
        r.sample()
        r.step(11)
        ref11 = _results(F, r, p)
    with F.Run(p, c1_tables) as r:
        r.run_graph(20)
        r.step(17)
        _same(_results(F, r, p), ref37)
        r.run_graph(11)
        _same(_results(F, r, p), ref11)
        r.sample()
        r.step(20)
        r.step(17)
        _same(_results(F, r, p), ref37)
        r.run_graph(11)
        _same(_results(F, r, p), ref11)


def test_refusals(F, inputs, c1_tables):
    p = inputs.config("c1_32", n_part=1000, n_grid=16, n_steps=8, precision=1)
    with F.Run(p, c1_tables) as r:
        for n in (-1, 9):
            with pytest.raises(F.FdfError) as e:
                r.run_graph(n)
            assert e.value.code == F.FDF_EINVAL
        F.fdf_timing(r.ctx, True)
        with pytest.raises(F.FdfError) as e:
            r.run_graph(8)
        assert e.value.code == F.FDF_ESTATE
        F.fdf_timing(r.ctx, False)
        r.set_fields(inputs.uniform_fields(p["n_grid"], np.ones(3) * 1e-6, np.zeros(3), 0.0, 0.0))
        with pytest.raises(F.FdfError) as e:
            r.run_graph(8)
        assert e.value.code == F.FDF_ESTATE
        r.set_fields(None)
        r.run_graph(0)
        assert r.state()[0] == 0
        r.step(8)
        assert r.state()[0] == 8
