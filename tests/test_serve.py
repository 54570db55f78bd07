"""Request server (include/igs_serve.h): each request against the CPU oracle, gangs of several
CTAs, the same result alone and in a mix, admission by device memory, the queue limit.

Tolerances as in the batched and precision forms: converged FP64 requests have the oracle's
status, step counts within +-2 and x within 1e-8 (relative); FP32-IR requests reach
beta <= tol with x within 1e-10 of the oracle's FP64 solution at tol = 1e-14.
"""
import ctypes as C
import time

import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def pkg():
    import paper_2205_07805_gb300 as pkg
    from paper_2205_07805_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _cases():
    out = []
    for i, (side, pe) in enumerate([(20, 1.0), (33, 40.0), (48, 90.0), (63, 10.0)]):
        A, b, _, _ = gen.cd2d(side, pe, seed=30 + i)
        out.append((A, b))
    for A, b, _, _ in gen.banded_batch(count=3, nmin=300, nmax=3000, seed=31):
        out.append((A, b))
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("rows_per_cta", [4096, 256])
def test_served_requests_match_oracle(pkg, rows_per_cta):
    """rows_per_cta = 256 puts every request but the smallest on a gang of several CTAs."""
    cases = _cases()
    norms = [gen.norm2_power(A, iters=100) for A, _ in cases]
    with pkg.Server(max_restart_m=40, arena_bytes=1 << 30, slots=3, rows_per_cta=rows_per_cta) as sv:
        ids = [sv.submit(A, b, A_norm2=nA, m=40, gs=2, tol=1e-12, max_restarts=200)
               for (A, b), nA in zip(cases, norms)]
        done = {c["id"]: c for c in sv.run_all()}
        for rid, (A, b), nA in zip(ids, cases, norms):
            c = done[rid]
            o = oracle.gmres(A, b, m=40, gs=2, tol=1e-12, max_cycles=200, normA=nA)
            x = sv.take(rid)
            assert c["status"] == o["status"] == 0, (c, o["status"])
            assert abs(c["steps"] - o["steps"]) <= 2, (c["steps"], o["steps"])
            err = np.linalg.norm(x - o["x"]) / np.linalg.norm(o["x"])
            assert err <= 1e-8, (A.n, c["gang_ctas"], err)
            if rows_per_cta == 256 and A.n > 512:
                assert c["gang_ctas"] > 1


@pytest.mark.gpu
def test_served_fp32_ir_requests(pkg):
    cases = _cases()[:3]
    norms = [gen.norm2_power(A, iters=100) for A, _ in cases]
    with pkg.Server(max_restart_m=60, arena_bytes=1 << 30, slots=3, rows_per_cta=512) as sv:
        ids = [sv.submit(A, b, A_norm2=nA, m=60, gs=2, tol=1e-14, max_restarts=100, precision="fp32_ir")
               for (A, b), nA in zip(cases, norms)]
        done = {c["id"]: c for c in sv.run_all()}
        for rid, (A, b), nA in zip(ids, cases, norms):
            o = oracle.gmres(A, b, m=60, gs=2, tol=1e-14, max_cycles=100, normA=nA)
            x = sv.take(rid)
            assert done[rid]["status"] == 0 and done[rid]["beta"] <= 1e-14
            assert np.linalg.norm(x - o["x"]) <= 1e-10 * np.linalg.norm(o["x"])


@pytest.mark.gpu
def test_same_result_alone_and_in_a_mix(pkg):
    A, b, _, _ = gen.cd2d(70, 30.0, seed=40)             # n = 4900: a gang of 10 at 512 rows
    nA = gen.norm2_power(A, iters=60)
    others = _cases()
    with pkg.Server(max_restart_m=50, arena_bytes=1 << 30, slots=1, rows_per_cta=512) as sv:
        rid = sv.submit(A, b, A_norm2=nA, m=50, tol=1e-12, max_restarts=100)
        alone = {c["id"]: c for c in sv.run_all()}[rid]
        x_alone = sv.take(rid)
    with pkg.Server(max_restart_m=50, arena_bytes=1 << 30, slots=4, rows_per_cta=512) as sv:
        ids = []
        for i, (Ao, bo) in enumerate(others):
            ids.append(sv.submit(Ao, bo, m=50, tol=1e-10 if i % 2 else 1e-12, max_restarts=100,
                                 precision="fp32_ir" if i % 3 == 0 else "fp64"))
            if i == 3:
                rid = sv.submit(A, b, A_norm2=nA, m=50, tol=1e-12, max_restarts=100)
            sv.pump()
        mixed = {c["id"]: c for c in sv.run_all()}[rid]
        x_mix = sv.take(rid)
    assert np.array_equal(x_alone, x_mix)
    assert alone["steps"] == mixed["steps"] and alone["beta"] == mixed["beta"]
    assert alone["gang_ctas"] == mixed["gang_ctas"] > 1


@pytest.mark.gpu
def test_admission_by_device_memory_and_queue_limit(pkg):
    cases = _cases()[:4]
    # an arena that holds the largest request but not two of them
    with pkg.Server(max_restart_m=40, arena_bytes=1 << 30, slots=4) as probe:
        rid = probe.submit(*cases[3], m=40)
        need = max(c["device_bytes"] for c in probe.run_all())
    with pkg.Server(max_restart_m=40, arena_bytes=int(need * 1.5), slots=4, max_queue=3) as sv:
        ids = [sv.submit(A, b, m=40, tol=1e-12, max_restarts=100) for A, b in cases[:3]]
        assert all(i is not None for i in ids)
        assert sv.submit(*cases[3], m=40) is None             # the queue is full
        done = sv.run_all()
        st = sv.stats()
        assert st["arena_peak"] <= st["arena_bytes"]
        assert len(done) == 3 and all(c["status"] == 0 for c in done)


@pytest.mark.gpu
def test_numeric_error_is_isolated(pkg):
    cases = _cases()[:3]
    with pkg.Server(max_restart_m=40, arena_bytes=1 << 30, slots=3, rows_per_cta=512) as sv:
        bad = cases[1][1].copy()
        bad[5] = np.nan
        ids = [sv.submit(cases[0][0], cases[0][1], m=40), sv.submit(cases[1][0], bad, m=40),
               sv.submit(cases[2][0], cases[2][1], m=40)]
        done = {c["id"]: c for c in sv.run_all()}
    assert done[ids[1]]["status"] == pkg.ENUMERIC
    assert done[ids[0]]["status"] == 0 and done[ids[2]]["status"] == 0


@pytest.mark.gpu
@pytest.mark.parametrize("lanes", [1, 3])
def test_graph_lane_requests_match_oracle_and_mix(pkg, lanes):
    """Requests with n >= graph_min_n run on the graph lanes (the whole-GPU kernels of igs.h,
    on the server's worker threads; with 3 lanes the three large requests run at once) beside
    gang requests: FP64 against the oracle as above, FP32-IR to beta <= 1e-14, and the graph
    request bitwise the same alone (one lane) and in the mix."""
    big = [gen.cd2d(side, pe, seed=50 + k)[:2] for k, (side, pe) in enumerate([(52, 30.0), (56, 70.0)])]
    small = _cases()[:3]
    norms_big = [gen.norm2_power(A, iters=100) for A, _ in big]
    norms_small = [gen.norm2_power(A, iters=100) for A, _ in small]
    gmin = 2500                   # the two grids (n = 2704, 3136); the small cases have n <= 2304
    with pkg.Server(max_restart_m=40, arena_bytes=1 << 30, slots=3, rows_per_cta=512, graph_min_n=gmin,
                    graph_lanes=lanes) as sv:
        ids_b = [sv.submit(A, b, A_norm2=nA, m=40, gs=2, tol=1e-12, max_restarts=200)
                 for (A, b), nA in zip(big, norms_big)]
        id_f = sv.submit(big[0][0], big[0][1], A_norm2=norms_big[0], m=40, gs=2, tol=1e-14, max_restarts=100,
                         precision="fp32_ir")
        ids_s = [sv.submit(A, b, A_norm2=nA, m=40, gs=2, tol=1e-12, max_restarts=200)
                 for (A, b), nA in zip(small, norms_small)]
        done = {c["id"]: c for c in sv.run_all()}
        xs = {rid: sv.take(rid) for rid in ids_b + [id_f] + ids_s}
    for rid, (A, b), nA in zip(ids_b, big, norms_big):
        c = done[rid]
        assert c["path"] == 1 and c["gang_ctas"] == 0 and c["A_norm2"] == nA
        o = oracle.gmres(A, b, m=40, gs=2, tol=1e-12, max_cycles=200, normA=nA)
        assert c["status"] == o["status"] == 0 and abs(c["steps"] - o["steps"]) <= 2, (c, o["steps"])
        assert np.linalg.norm(xs[rid] - o["x"]) <= 1e-8 * np.linalg.norm(o["x"])
    c = done[id_f]
    o = oracle.gmres(big[0][0], big[0][1], m=40, gs=2, tol=1e-14, max_cycles=100, normA=norms_big[0])
    assert c["path"] == 1 and c["status"] == 0 and c["beta"] <= 1e-14
    assert np.linalg.norm(xs[id_f] - o["x"]) <= 1e-10 * np.linalg.norm(o["x"])
    for rid in ids_s:
        assert done[rid]["path"] == 0 and done[rid]["status"] == 0
    with pkg.Server(max_restart_m=40, arena_bytes=1 << 30, slots=1, rows_per_cta=512, graph_min_n=gmin) as sv:
        rid = sv.submit(big[1][0], big[1][1], A_norm2=norms_big[1], m=40, gs=2, tol=1e-12, max_restarts=200)
        alone = {c["id"]: c for c in sv.run_all()}[rid]
        x_alone = sv.take(rid)
    assert alone["steps"] == done[ids_b[1]]["steps"] and alone["beta"] == done[ids_b[1]]["beta"]
    assert np.array_equal(x_alone, xs[ids_b[1]])


@pytest.mark.gpu
def test_server_estimates_norm_when_not_given(pkg):
    """A request without ||A||_2 gets the library's GPU power-iteration estimate (gang path:
    the server's norm worker; graph lane: the lane's igs_create), so beta is eq. "nrbe" with
    ||A||_2 estimated from below (within 1% of the SVD value here), not the larger bound
    sqrt(||A||_1 ||A||_inf); the completion record carries it and the oracle's beta of the
    returned x with that norm meets the tolerance."""
    small = [gen.cd2d(side, pe, seed=70 + k)[:2] for k, (side, pe) in enumerate([(30, 10.0), (40, 80.0)])]
    big = gen.cd2d(52, 40.0, seed=75)[:2]
    with pkg.Server(max_restart_m=40, arena_bytes=1 << 30, slots=2, rows_per_cta=512, graph_min_n=2500) as sv:
        ids = [sv.submit(A, b, m=40, gs=2, tol=1e-12, max_restarts=200) for A, b in small + [big]]
        done = {c["id"]: c for c in sv.run_all()}
        xs = {rid: sv.take(rid) for rid in ids}
    for rid, (A, b) in zip(ids, small + [big]):
        c = done[rid]
        D = gen.csr_to_dense(A)
        s2 = float(np.linalg.norm(D, 2))
        bound = float(np.sqrt(np.abs(D).sum(0).max() * np.abs(D).sum(1).max()))
        assert 0.99 * s2 <= c["A_norm2"] <= s2 * (1 + 1e-12), (c["A_norm2"], s2)
        assert c["A_norm2"] < bound
        assert c["status"] == 0 and c["beta"] <= 1e-12
        assert oracle.backward_error(A, b, xs[rid], c["A_norm2"]) <= 1e-12
    assert done[ids[-1]]["path"] == 1 and all(done[r]["path"] == 0 for r in ids[:-1])


@pytest.mark.gpu
def test_gang_wait_runs_out_without_a_fault(pkg):
    """The gangs' bounded waits: with the arrival counter started where no arrival completes
    the barrier (a flag nothing sets), every CTA's wait gives up, the gang's abort flag is
    raised and the call reports IGS_ETIMEOUT; the device then still runs gangs and solves."""
    lib = pkg.load_library()
    ab = C.c_int(-1)
    assert lib.igs_server_gang_selftest(0, 8, 0, C.byref(ab)) == 0 and ab.value == 0
    t0 = time.perf_counter()
    assert lib.igs_server_gang_selftest(0, 8, 1, C.byref(ab)) == -5 and ab.value == 1
    waited = time.perf_counter() - t0
    print(f"stalled gang gave up after {waited:.2f} s")
    assert waited < 30.0
    assert lib.igs_server_gang_selftest(0, 8, 0, C.byref(ab)) == 0 and ab.value == 0
    A, b, _, _ = gen.cd2d(40, 20.0, seed=60)
    with pkg.Server(max_restart_m=30, arena_bytes=1 << 28, slots=1, rows_per_cta=512) as sv:
        rid = sv.submit(A, b, m=30, tol=1e-12, max_restarts=100)
        c = {c["id"]: c for c in sv.run_all()}[rid]
        sv.take(rid)
    assert c["status"] == 0 and c["gang_ctas"] > 1


@pytest.mark.gpu
def test_served_full_size_requests(pkg):
    """Requests of the served benchmark's largest sizes: a 1024 x 1024 grid (n = 1,048,576)
    on the graph lane in FP64 and a 700 x 700 grid (n = 490,000) on a gang of 120 CTAs in
    FP32-IR, both to beta <= 1e-10; beta is recomputed by the oracle from the returned x
    with the server's norm bound sqrt(||A||_1 ||A||_inf)."""
    reqs = [(gen.cd2d(1024, 60.0, seed=70)[:2], "fp64"), (gen.cd2d(700, 30.0, seed=71)[:2], "fp32_ir")]
    with pkg.Server(max_restart_m=100, arena_bytes=8 << 30, slots=2, rows_per_cta=4096,
                    graph_min_n=1_000_000) as sv:
        ids = [sv.submit(A, b, m=100, gs=2, tol=1e-10, max_restarts=2000, precision=prec)
               for (A, b), prec in reqs]
        done = {c["id"]: c for c in sv.run_all()}
        xs = [sv.take(rid) for rid in ids]
    for rid, x, ((A, b), prec) in zip(ids, xs, reqs):
        c = done[rid]
        assert c["status"] == 0 and c["beta"] <= 1e-10, c
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        av = np.abs(A.val)
        bound = float(np.sqrt(np.bincount(A.colind, av, A.n).max() * np.bincount(rows, av, A.n).max()))
        beta_o = oracle.backward_error(A, b, x, bound)
        print(f"n={A.n} {prec} path {c['path']} G={c['gang_ctas']}: {c['steps']} steps, beta {c['beta']:.2e}, "
              f"oracle beta {beta_o:.2e}")
        assert beta_o <= 1e-10 * (1 + 1e-6)
    assert done[ids[0]]["path"] == 1 and done[ids[1]]["path"] == 0 and done[ids[1]]["gang_ctas"] == 120
