"""The serving layer on the GPU (include/tf_server.h), through the C ABI: factorisation
jobs of mixed sizes admitted against device memory and run concurrently, fold-in
requests batched continuously against a model, and the same result for every job and
every fold-in alone and in the mix (bit for bit: contexts share no device state and a
fold-in's partial sums follow its own fixed order).  Also the memory estimate against
the pool's measured high-water mark."""
import numpy as np
import pytest

import paper_1410_5209_gb300 as tf
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_5209_gb300 import build
    build.build()


def job_problems():
    # mixed sizes and shapes; C = 4 (narrow path) and C = 20 (wide path), float and double
    spec = [((400, 300, 60), 40_000, 16, 4, tf.F32), ((1200, 90, 40), 25_000, 16, 4, tf.F32),
            ((300, 250, 80), 60_000, 24, 20, tf.F32), ((150, 120, 30, 20), 30_000, 12, 4, tf.F64),
            ((900, 800, 50), 80_000, 16, 8, tf.F32), ((200, 200, 200), 10_000, 16, 16, tf.F64)]
    out = []
    for i, (dims, nnz, K, C, dt) in enumerate(spec):
        p = synth.small(300 + i, dims, nnz, 4, K)
        out.append((p, C, dt))
    return out


def solo(p, C, dt, sweeps, lam):
    c, x = p.numpy()
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=dt)
    for s in range(sweeps):
        f.sweep(C, lam, 1, p.column_order(s, C))
    res = [f.factors(n) for n in range(p.N)], f.loss(lam)
    f.close()
    return res


def orders(p, C, sweeps):
    return np.stack([p.column_order(s, C) for s in range(sweeps)]).astype(np.int32)


def test_estimate_bounds_the_pool_high_water():
    p = synth.small(320, (3000, 2000, 100), 400_000, 4, 48)
    c, x = p.numpy()
    used0, _, _ = tf.pool_usage(reset_high=True)
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32)
    for C, s in ((10, 0), (40, 1)):
        f.sweep(C, 0.1, 1, p.column_order(s, C))
    f.loss(0.1)
    f.sync()
    _, high, _ = tf.pool_usage()
    est = tf.estimate_bytes(p.dims, p.nnz, p.K, 40, tf.F32)
    grew = high - used0
    f.close()
    assert 0 < grew <= est, (grew, est)
    assert est <= 2.5 * grew, (grew, est)


def test_jobs_and_foldins_in_the_mix_match_solo_runs():
    lam, sweeps = 0.2, 3
    probs = job_problems()
    expect = [solo(p, C, dt, sweeps, lam) for p, C, dt in probs]

    mp = synth.small(330, (2000, 500, 80), 120_000, 4, 32)
    mc, mx = mp.numpy()
    model = tf.Factorization(mc, mx, mp.dims, mp.K, seed=mp.seed, dtype=tf.F32)
    model.sweep(8, lam, 1)
    reqs = synth.foldin_requests(mp, 60, 331, m_min=5, m_max=3000)
    alone = [model.foldin_batch(0, [r], lam) for r in reqs]

    srv = tf.Server(model, max_running=3, max_batch=16)
    ids = [srv.submit_job(*p.numpy(), p.dims, p.K, C, lam, sweeps, seed=p.seed, dtype=dt,
                          orders=orders(p, C, sweeps)) for p, C, dt in probs]
    rids = [srv.submit_foldin(0, o, v, lam) for o, v in reqs]
    got = [srv.wait_foldin(r) for r in rids]
    infos = [srv.wait_job(j) for j in ids]
    for (p, C, dt), j, info, (fa, la) in zip(probs, ids, infos, expect):
        assert info["state"] == tf.JOB_DONE, info
        assert info["sweeps_done"] == sweeps
        assert (info["loss"], info["rmse"]) == la
        for n in range(p.N):
            assert np.array_equal(srv.job_factors(j, n), fa[n])
        srv.release_job(j)
    for (row, st, lat), (rows_a, st_a) in zip(got, alone):
        assert st == st_a[0] == 0
        assert np.array_equal(row, rows_a[0])
        assert lat > 0
    s = srv.stats()
    assert s["jobs_done"] == len(probs) and s["jobs_failed"] == 0
    assert s["foldins_done"] == len(reqs)
    assert 1 <= s["running_peak"] <= 3
    assert s["bytes_admitted"] == 0
    srv.close()
    # the model is back on its own stream and usable
    assert np.array_equal(model.foldin_batch(0, [reqs[0]], lam)[0], alone[0][0])


def test_budget_serialises_jobs():
    """A budget that holds one job at a time: jobs run one after another, never more
    admitted bytes than the budget, and all finish."""
    lam, sweeps = 0.2, 2
    probs = [(synth.small(340 + i, (300, 250, 80), 60_000, 4, 24), 20, tf.F32)
             for i in range(3)]
    need = [tf.estimate_bytes(p.dims, p.nnz, p.K, C, dt) for p, C, dt in probs]
    budget = max(need)
    assert sum(sorted(need)[:2]) > budget   # no two of them fit together
    srv = tf.Server(hbm_budget=budget, max_running=4)
    ids = [srv.submit_job(*p.numpy(), p.dims, p.K, C, lam, sweeps, seed=p.seed, dtype=dt)
           for p, C, dt in probs]
    for j in ids:
        info = srv.wait_job(j)
        assert info["state"] == tf.JOB_DONE
        srv.release_job(j)
    s = srv.stats()
    assert s["bytes_admitted_peak"] <= budget
    assert s["running_peak"] == 1
    srv.close()


def test_refusals_and_shutdown():
    p, C, dt = job_problems()[0]
    srv = tf.Server(hbm_budget=1 << 20, max_running=1)
    with pytest.raises(tf.TFError) as e:   # larger than the whole budget: never admissible
        srv.submit_job(*p.numpy(), p.dims, p.K, C, 0.1, 1, seed=p.seed)
    assert e.value.status == tf.ENOMEM
    with pytest.raises(tf.TFError) as e:   # no model: no fold-ins
        srv.submit_foldin(0, np.zeros((1, 2), np.int32), np.zeros(1, np.float32), 0.1)
    assert e.value.status == tf.EINVAL
    srv.close()

    # jobs still queued at shutdown fail with TF_EBUSY; nothing hangs
    srv = tf.Server(max_running=1)
    ids = [srv.submit_job(*p.numpy(), p.dims, p.K, C, 0.1, 20, seed=p.seed) for _ in range(4)]
    with pytest.raises(tf.TFError) as e:   # bad col_orders row
        srv.submit_job(*p.numpy(), p.dims, p.K, C, 0.1, 1, seed=p.seed,
                       orders=np.zeros((1, p.K), np.int32))
    assert e.value.status == tf.EINVAL
    info = srv.job_info(ids[-1])
    assert info["state"] in (tf.JOB_QUEUED, tf.JOB_RUNNING, tf.JOB_DONE)
    srv.close()


def test_pool_keeps_freed_memory_until_trimmed():
    """A destroyed context's memory stays in the library's pool (the next context of the
    same size takes it without growing the pool); tf_pool_trim hands it back."""
    p = synth.small(350, (3000, 2000, 100), 300_000, 4, 16)
    c, x = p.numpy()
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32)
    f.sweep(4, 0.1, 1)
    f.sync()
    used1, _, held1 = tf.pool_usage()
    f.close()
    import torch
    torch.cuda.synchronize()   # the frees run in stream order
    used2, _, held2 = tf.pool_usage()
    assert used2 < used1 and held2 >= held1 - (1 << 21)
    g = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32)
    g.sweep(4, 0.1, 1)
    g.sync()
    _, _, held3 = tf.pool_usage()
    assert held3 <= held2 + (8 << 20)   # reused, not grown (up to pool rounding)
    g.close()
    tf.pool_trim(0)
    used4, _, held4 = tf.pool_usage()
    assert held4 <= used4 + (2 << 20)
