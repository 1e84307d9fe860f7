"""Host-only logic of the serving layer, no GPU: the admission decision of the
scheduler (first fit in arrival order, a bound on how often a job may be passed, the
budget and slot limits) on hand-worked cases, and the device-memory estimate against
the sizes it must at least cover."""
import numpy as np
import pytest

import paper_1410_5209_gb300 as tf


@pytest.fixture(scope="module", autouse=True)
def lib():
    try:
        return tf.load()
    except tf.LibraryMissing:
        from paper_1410_5209_gb300 import build
        build.build()
        return tf.load()


def test_first_fit_in_arrival_order():
    # room 6: job 0 (5) starts; job 1 (3) and job 2 (8) do not fit; job 3 (1) does and
    # passes jobs 1 and 2 once each
    admit, byp = tf.plan_admission([5, 3, 8, 1], [0, 0, 0, 0], room=6)
    assert admit.tolist() == [True, False, False, True]
    assert byp.tolist() == [0, 1, 1, 0]


def test_job_passed_too_often_holds_the_queue():
    # job 0 has been passed max_bypass times: nothing behind it starts until it fits
    admit, byp = tf.plan_admission([9, 1, 1], [8, 0, 0], room=4, max_bypass=8)
    assert not admit.any()
    assert byp.tolist() == [8, 0, 0]
    admit, _ = tf.plan_admission([9, 1, 1], [8, 0, 0], room=9, max_bypass=8)
    assert admit.tolist() == [True, False, False]


def test_strict_arrival_order():
    admit, byp = tf.plan_admission([5, 1, 1], [0, 0, 0], room=4, max_bypass=-1)
    assert not admit.any() and byp.tolist() == [0, 0, 0]
    admit, _ = tf.plan_admission([2, 1, 9, 1], [0, 0, 0, 0], room=20, max_bypass=-1)
    assert admit.tolist() == [True, True, True, True]


def test_budget_and_slots():
    # the budget binds before the room does
    admit, _ = tf.plan_admission([4, 4, 4], [0, 0, 0], room=100, budget_left=9)
    assert admit.tolist() == [True, True, False]
    # two slots: the third job waits even though it fits
    admit, byp = tf.plan_admission([1, 1, 1], [0, 0, 0], room=100, slots=2)
    assert admit.tolist() == [True, True, False]
    assert byp.tolist() == [0, 0, 0]
    # a job exactly as large as the room fits
    admit, _ = tf.plan_admission([7], [0], room=7)
    assert admit.tolist() == [True]
    # empty queue
    admit, byp = tf.plan_admission(np.zeros(0, np.int64), np.zeros(0, np.int32), room=7)
    assert admit.size == 0


def test_estimate_covers_the_resident_arrays():
    """The estimate is at least what a context keeps resident: values, N residual copies,
    N sorted orders, N(N-1) other-mode index streams, the factors, and for float
    three-way tensors the lean pass's gather plans (a location word per entry and mode)."""
    dims, nnz, K = (100_000, 100_000, 1_000), 100_000_000, 100
    est = tf.estimate_bytes(dims, nnz, K, 10, tf.F32, num_sms=152)
    N = 3
    resident = nnz * 4 * (1 + N + N + N * (N - 1) + N) + sum(dims) * K * 4
    assert resident <= est <= 1.5 * resident
    # and at least the layout build's peak: values, SoA coordinates, a key array and the
    # sort's two alternate arrays beside the per-mode orders and index streams
    build = nnz * 4 * (1 + N + 1 + 2 + N + N * (N - 1))
    assert est >= build


def test_estimate_grows_with_the_problem():
    base = dict(dims=(5000, 4000, 300), nnz=2_000_000, K=32, C_max=8, num_sms=152)
    e0 = tf.estimate_bytes(base["dims"], base["nnz"], base["K"], base["C_max"],
                           num_sms=152)
    assert tf.estimate_bytes(base["dims"], 4_000_000, 32, 8, num_sms=152) > e0
    assert tf.estimate_bytes(base["dims"], 2_000_000, 64, 8, num_sms=152) > e0
    assert tf.estimate_bytes(base["dims"], 2_000_000, 32, 30, num_sms=152) > e0
    # wider values (four-way, where neither dtype has gather plans)
    d4 = (5000, 4000, 300, 20)
    assert tf.estimate_bytes(d4, 2_000_000, 32, 8, tf.F64, num_sms=152) > \
        tf.estimate_bytes(d4, 2_000_000, 32, 8, tf.F32, num_sms=152)
    # device-resident input needs no host-copy staging
    assert tf.estimate_bytes(base["dims"], 2_000_000, 32, 8, device_input=True,
                             num_sms=152) <= e0


@pytest.mark.parametrize("args", [
    ((10, 10), 100, 4, 5),       # C > K
    ((10, 10), 100, 4, 0),       # C < 1
    ((10, 0), 100, 4, 2),        # empty mode
    ((10, 10), -1, 4, 2),        # negative nnz
    ((10,) * 9, 100, 4, 2),      # N > 8
    ((10, 10), 100, 200, 150),   # C >= 128
])
def test_estimate_rejects_what_create_or_sweep_refuse(args):
    dims, nnz, K, C = args
    with pytest.raises(tf.TFError) as e:
        tf.estimate_bytes(dims, nnz, K, C, num_sms=152)
    assert e.value.status == tf.EINVAL
