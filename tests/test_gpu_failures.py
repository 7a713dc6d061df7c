"""Failure detection on the GPU without faulting it: every error status of
the C ABI is produced by a host-side or data-side condition (bad arguments,
missing set-up, non-finite data, step-size underflow, no convergence), a
device wait that runs out is reported as MM_ETIMEOUT with the context still
usable, and a failing request in a batch fails alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _state(n=(8, 6, 2), prec="fp64", m=None):
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import to_soa
    s = State(n, (3e-9, 3e-9, 3e-9), prec)
    s.set_material(Ms=8e5, A=1.3e-11, alpha=0.5)
    s.demag_setup()
    if m is not None:
        s.set_m(to_soa(m))
    return s


def _status(exc):
    from paper_2302_08843_gb300 import binding
    return binding.STATUS_NAMES[exc.value.status]


def _rand_m(n, seed=0):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=n + (3,))
    return m / np.linalg.norm(m, axis=-1, keepdims=True)


def test_invalid_arguments():
    from paper_2302_08843_gb300.binding import Batch, MMError, State
    with pytest.raises(MMError) as e:
        State((0, 4, 4), (1e-9, 1e-9, 1e-9), "fp64")
    assert _status(e) == "MM_EINVAL"
    s = _state(m=_rand_m((8, 6, 2)))
    with pytest.raises(MMError) as e:
        s.step(-1e-13)
    assert _status(e) == "MM_EINVAL"
    s.close()
    b = Batch((8, 8, 1), (3e-9,) * 3, "fp32", capacity=2)
    with pytest.raises(MMError) as e:
        b.set_slot(5, 8e5, 1e-11, 1.0, np.zeros((3, 1, 8, 8), np.float32))
    assert _status(e) == "MM_EINVAL"
    with pytest.raises(MMError) as e:
        b.begin(0)
    assert _status(e) == "MM_EINVAL"
    b.close()


def test_not_set_up():
    from paper_2302_08843_gb300.binding import MMError
    s = _state()
    with pytest.raises(MMError) as e:
        s.step(1e-13)
    assert _status(e) == "MM_ENOTSETUP"
    s.close()


def test_non_finite_magnetisation():
    from paper_2302_08843_gb300.binding import MMError
    m = _rand_m((8, 6, 2))
    m[3, 2, 1] = np.nan
    s = _state(m=m)
    with pytest.raises(MMError) as e:
        s.heff(torque=True)
    assert _status(e) == "MM_ENONFINITE"
    s.close()


def test_step_size_underflow():
    from paper_2302_08843_gb300.binding import MMError
    s = _state(m=_rand_m((8, 6, 2), 1))
    with pytest.raises(MMError) as e:
        s.step(1e-13, 0.0, "dp45", rtol=1e-300)     # no step can meet this tolerance
    assert _status(e) == "MM_ESTEP"
    s.close()


def test_not_converged():
    from paper_2302_08843_gb300.binding import MMError
    s = _state(m=_rand_m((8, 6, 2), 2))
    with pytest.raises(MMError) as e:
        s.relax(tol=1e-12, max_steps=3)
    assert _status(e) == "MM_ENOTCONVERGED"
    s.close()


def test_device_wait_runs_out_and_context_survives():
    from paper_2302_08843_gb300.binding import MMError
    m = _rand_m((8, 6, 2), 3)
    s = _state(m=m)
    h_ref, E_ref = s.heff(energies=True)
    s.selftest_wait_timeout(1 << 16)
    with pytest.raises(MMError) as e:
        s.heff(energies=True)
    assert _status(e) == "MM_ETIMEOUT"
    s.close()
    # the context is intact: a new state computes the same field
    s2 = _state(m=m)
    h2, E2 = s2.heff(energies=True)
    assert np.array_equal(h2.cpu().numpy(), h_ref.cpu().numpy()) and E2 == E_ref
    s2.close()


def test_failing_request_fails_alone_in_a_batch():
    from paper_2302_08843_gb300.binding import Batch
    from paper_2302_08843_gb300.workloads import to_soa
    n = (12, 8, 2)
    good = _rand_m(n, 4)
    bad = _rand_m(n, 5)
    bad[0, 0, 0] = np.inf
    outs = []
    for with_bad in (False, True):
        b = Batch(n, (3e-9,) * 3, "fp32", capacity=3)
        b.set_slot(0, 8e5, 1.3e-11, 1.0, to_soa(good).astype(np.float32))
        if with_bad:
            b.set_slot(1, 8e5, 1.3e-11, 1.0, to_soa(bad).astype(np.float32))
        while True:
            b.begin(8, 1e-5, 1e-3, 5000)
            st, steps, tq = b.end()
            if not np.any(st == 1):
                break
        outs.append((st.copy(), steps.copy(), b.get_m(0)))
        b.close()
    assert outs[1][0][1] == 4                      # the bad request failed
    assert outs[0][0][0] == outs[1][0][0] == 2     # the good one converged both times
    assert outs[0][1][0] == outs[1][1][0]
    assert np.array_equal(outs[0][2], outs[1][2])  # bitwise the same as alone
