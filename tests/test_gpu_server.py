"""The request server (fdf_server_*): continuous batching of independent runs.

Every neutrino is independent once the metric is known (Sec. 2.1), so every
run is too: a request's results must not depend on what else shares the GPU.
These tests run requests of different grid sizes, particle counts, species
counts, masses and step counts alone and in a mix, and compare:

* positions, momenta and weights bitwise (each particle's arithmetic is the
  same, whatever the sort order or the neighbouring streams);
* the deposit to 1e-12 relative to its largest cell (FP64 atomic additions in
  another order).

They also check one request against the oracle at the parity tolerances,
admission by footprint against the arena budget, and refusal of a request
larger than the whole budget.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

GiB = 1 << 30


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


def _mix(inputs):
    return [
        inputs.config("c2_128", n_part=20000, n_grid=32, n_species=2, m_ev=[0.05, 0.2], n_steps=23, seed=71,
                      precision=1),
        inputs.config("c2_128", n_part=33 ** 3, n_grid=64, n_species=1, m_ev=[0.12], n_steps=17, seed=72,
                      precision=1),
        inputs.config("c2_128", n_part=5000, n_grid=16, n_species=3, m_ev=[0.02, 0.1, 0.3], n_steps=31, seed=73,
                      precision=2),
        inputs.config("c2_128", n_part=7001, n_grid=16, n_species=2, m_ev=[0.04, 0.15], n_steps=19, seed=75,
                      precision=3),
        inputs.config("c2_128", n_part=4096, n_grid=32, n_species=1, m_ev=[0.08], n_steps=12, seed=74,
                      precision=0),
    ]


def _results(F, srv, rid):
    out = []
    for s in range(srv.params[rid]["n_species"]):
        out.append(srv.get(rid, s))
    return out, srv.deposit(rid)


@pytest.mark.parametrize("merge", [False, True], ids=["streams", "merged"])
def test_each_request_is_the_same_alone_and_in_the_mix(F, inputs, merge):
    """With merged passes the FP64-state requests of the mix share launches (the FP32 and
    the BF16 ones separately); the split-state and plain FP64 requests keep their own."""
    reqs = _mix(inputs)
    tables = inputs.transfer_tables(reqs[0])
    alone = []
    with F.Server(4 * GiB, max_active=1, slice_steps=5, merge=merge) as srv:
        for p in reqs:
            rid = srv.submit(p, tables)
            assert srv.wait(120000) == rid
            info = srv.info(rid)
            assert info.status == F.FDF_REQ_DONE, info.message
            alone.append(_results(F, srv, rid))
            srv.release(rid)
    with F.Server(4 * GiB, max_active=5, slice_steps=5, merge=merge) as srv:
        ids = [srv.submit(p, tables) for p in reqs[:-1]]
        # one request arrives while the others are on the GPU
        got = srv.wait(120000)
        ids.append(srv.submit(reqs[-1], tables))
        finished = {got}
        while len(finished) < len(ids):
            r = srv.wait(120000)
            assert r is not None
            finished.add(r)
        for p, rid, ref in zip(reqs, ids, alone):
            info = srv.info(rid)
            assert info.status == F.FDF_REQ_DONE, info.message
            assert info.t_submit <= info.t_admit <= info.t_done
            parts, dep = _results(F, srv, rid)
            for s, ((x, q, w), (x0, q0, w0)) in enumerate(zip(parts, ref[0])):
                assert np.array_equal(x, x0) and np.array_equal(q, q0) and np.array_equal(w, w0), (rid, s)
            scale = np.max(np.abs(ref[1]))
            err = np.max(np.abs(dep - ref[1])) / scale
            print("request %d: deposit alone vs mix %.2e of max cell" % (rid, err))
            assert err <= 1e-12
            srv.release(rid)
        if merge:
            print("merged launches:", srv.merged_launches())
            assert srv.merged_launches() > 0


@pytest.mark.parametrize("merge", [False, True], ids=["streams", "merged"])
def test_server_result_matches_the_oracle(F, inputs, merge):
    p = inputs.config("c1_32", n_part=3000, n_grid=16, n_steps=20, precision=1, seed=77)
    tables = inputs.transfer_tables(p)
    o = O.Oracle(p, tables)
    ref = o.run(np.arange(p["n_part"]))
    with F.Server(2 * GiB, max_active=2, slice_steps=3, merge=merge) as srv:
        rid = srv.submit(p, tables)
        assert srv.wait(120000) == rid
        assert srv.info(rid).status == F.FDF_REQ_DONE
        x, q, w = srv.get(rid, 0)
        srv.release(rid)
    L = p["box"]
    dx = np.abs(x - ref["x"])
    dx = np.minimum(dx, L - dx)
    qn = np.linalg.norm(ref["q"], axis=0)
    print("server vs oracle: x %.2e L, q %.2e, w %.2e" % (dx.max() / L, (np.abs(q - ref["q"]) / qn).max(),
                                                        np.abs(w - ref["w"]).max()))
    assert dx.max() <= 1e-6 * L
    assert (np.abs(q - ref["q"]) / qn).max() <= 1e-5
    assert np.abs(w - ref["w"]).max() <= 1e-5


def test_admission_waits_for_memory_and_refuses_oversize(F, inputs):
    p = inputs.config("c2_128", n_part=64 ** 3, n_grid=64, n_steps=10, precision=1, seed=78)
    tables = inputs.transfer_tables(p)
    need = F.fdf_footprint(F.make_params(p))
    budget = int(1.5 * need) + (4 << 20)   # room for one such request, not two
    with F.Server(budget, max_active=4, slice_steps=4) as srv:
        a = srv.submit(p, tables)
        b = srv.submit(dict(p, seed=79), tables)
        assert srv.wait(120000) == a
        # b cannot be admitted while a holds its memory
        assert srv.wait(300) is None
        assert srv.info(b).status == F.FDF_REQ_QUEUED
        assert srv.load()[0] == 1
        t_release = srv.clock()
        srv.release(a)
        assert srv.wait(120000) == b
        ib = srv.info(b)
        assert ib.status == F.FDF_REQ_DONE
        assert ib.t_admit >= t_release
        srv.release(b)
        assert srv.load() == (0, 0, 0)
        with pytest.raises(F.FdfError) as e:
            srv.submit(dict(p, n_part=512 ** 3), tables)
        assert e.value.code == F.FDF_ENOMEM
        with pytest.raises(F.FdfError) as e:
            srv.release(12345)
        assert e.value.code == F.FDF_EINVAL
