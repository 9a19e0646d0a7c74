"""The reconstruction server on the GPU (through the C ABI).

* Each job's result is the same alone and in a mix of concurrent jobs, bitwise, with
  batched clipping (the jobs' cells share one launch per pass) and without: a cell's
  arithmetic and a job's reductions never involve another job (integer atomics only,
  fixed-order reductions).
* Without batching a job runs exactly the single-box kernels, so its result equals the
  direct path (sdot_create + sdot_solve + sdot_displacement) bitwise; the batched
  kernel is another instantiation of the same cell code and is held to the solve's
  own accuracy.
* Admission keeps the admitted jobs' footprints within the budget; a job larger than
  the budget is refused; a job that fails reports its own error and leaves the others
  intact.
"""
import numpy as np
import pytest

from paper_2110_08868_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2110_08868_gb300 import binding as B  # noqa: E402


def _box(n, seed):
    y, _, _ = ics.zeldovich_box(n, 1.0, ics.spectrum_kinv, 0.3, seed)
    return np.ascontiguousarray(y)


JOBS = [(12, 1001), (16, 1002), (20, 1003), (14, 1004)]
TOL = 1e-6


def _run(jobs, max_active, one_at_a_time, batch_clip):
    srv = B.Server(max_active=max_active, batch_clip=batch_clip)
    out = {}
    try:
        if one_at_a_time:
            for n, seed in jobs:
                jid = srv.submit(_box(n, seed), [1.0] * 3, TOL)
                assert srv.wait(jid, 120.0)
                out[(n, seed)] = srv.result(jid)
        else:
            ids = {(n, seed): srv.submit(_box(n, seed), [1.0] * 3, TOL) for n, seed in jobs}
            for key, jid in ids.items():
                assert srv.wait(jid, 120.0)
                out[key] = srv.result(jid)
        info = srv.info()
    finally:
        srv.close()
    return out, info


@pytest.mark.parametrize("batch_clip", [True, False])
def test_same_alone_and_in_the_mix(batch_clip):
    alone, _ = _run(JOBS, 1, True, batch_clip)
    mixed, info = _run(JOBS, 8, False, batch_clip)
    assert info["finished"] == len(JOBS)
    for key in alone:
        a, m = alone[key], mixed[key]
        assert a["stats"]["max_rel_err"] <= TOL
        np.testing.assert_array_equal(a["disp"], m["disp"])
        np.testing.assert_array_equal(a["psi"], m["psi"])
        assert a["stats"]["newton_iters"] == m["stats"]["newton_iters"]
        assert a["stats"]["laguerre_evals"] == m["stats"]["laguerre_evals"]
        t = m["times"]
        assert t[0] <= t[1] <= t[2]


def test_server_equals_direct_path():
    n, seed = JOBS[2]
    y = _box(n, seed)
    a = 1.0 / n
    s = B.Solver(y, [1.0] * 3)
    st = s.solve(TOL)
    d = s.displacement()
    psi = s.psi()
    s.close()
    for batch_clip in (False, True):
        srv = B.Server(batch_clip=batch_clip)
        try:
            jid = srv.submit(y, [1.0] * 3, TOL)
            assert srv.wait(jid, 120.0)
            r = srv.result(jid)
        finally:
            srv.close()
        assert r["stats"]["max_rel_err"] <= TOL
        if not batch_clip:
            assert r["stats"]["newton_iters"] == st["newton_iters"]
            np.testing.assert_array_equal(r["disp"], d)
            np.testing.assert_array_equal(r["psi"], psi)
        else:
            # both solved to max|V - nu|/nu <= 1e-6: displacements agree to the
            # centroid shift such a volume error allows
            assert np.max(np.abs(r["disp"] - d)) <= 1e-4 * a


def test_admission_budget_and_failures():
    rc, fp_big = B.sdot_server_footprint(20 ** 3, [1.0] * 3)
    B.check(rc)
    budget = int(fp_big * 1.5)  # at most one 20^3 job at a time
    srv = B.Server(hbm_budget=budget, max_active=8)
    try:
        # a job that can never fit
        rc, _ = B.sdot_server_submit(srv.srv, _box(32, 7), None, [1.0] * 3, TOL,
                                     B.sdot_default_options())
        assert rc == B.SDOT_ERR_OOM
        # a job that fails on the device side (duplicate seeds) among good ones
        bad = _box(12, 8)
        bad[5] = bad[9]
        ids = [srv.submit(_box(20, 10 + t), [1.0] * 3, TOL) for t in range(3)]
        jbad = srv.submit(bad, [1.0] * 3, TOL)
        for jid in ids + [jbad]:
            assert srv.wait(jid, 120.0)
        with pytest.raises(B.SdotError) as e:
            srv.result(jbad)
        assert e.value.code == B.SDOT_ERR_DUPLICATE
        for jid in ids:
            assert srv.result(jid)["stats"]["max_rel_err"] <= TOL
        info = srv.info()
        assert info["peak_used_bytes"] <= budget
        assert info["used_bytes"] == 0 and info["active"] == 0
        assert info["finished"] == 4
    finally:
        srv.close()


@pytest.mark.parametrize("batch_clip", [True, False])
def test_server_job_matches_the_oracle(batch_clip):
    # a 12^3 job solved by the server (in a mix with two other jobs) to 1e-10, against
    # the oracle's own damped-Newton solve of the same box to 1e-11: the displacements
    # agree within 1e-6 lattice spacings (eq. laguerrecell at the unique solution)
    import sdot_oracle as O

    n, seed = 12, 1011
    y = _box(n, seed)
    a = 1.0 / n
    nu = ics.uniform_masses(y.shape[0], 1.0)
    srv = B.Server(max_active=4, batch_clip=batch_clip)
    try:
        others = [srv.submit(_box(m, s), [1.0] * 3, 1e-6) for m, s in ((16, 1012), (14, 1013))]
        jid = srv.submit(y, [1.0] * 3, 1e-10, precision="fp64")
        assert srv.wait(jid, 120.0)
        r = srv.result(jid)
        for o in others:
            assert srv.wait(o, 120.0)
            srv.result(o)
    finally:
        srv.close()
    assert r["stats"]["max_rel_err"] <= 1e-10
    _, info = O.solve(y, nu, 1.0, tol=1e-11)
    assert np.max(np.abs(r["disp"] - info["disp"])) <= 1e-6 * a
