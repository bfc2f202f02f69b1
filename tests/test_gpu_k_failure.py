"""Failure detection on the GPU without a fault: the bounded wait of the
tensor-core likelihood kernel runs out on a barrier that nothing completes,
reports through the device status word (FG21_E_DEVICE on the host), stops the
other waiting warps through the abort signal, and leaves the CUDA context
usable: a likelihood call right after it still matches the oracle."""
import numpy as np
import pytest

import cases
from conftest import report

pytestmark = pytest.mark.gpu

WAIT_LIMIT_S = 4.0


def test_bounded_wait_expires_reports_and_recovers(fg21lib):
    rc, status, elapsed = fg21lib.fg21_selftest_bounded_wait()
    report("bounded_wait_selftest", status=status, elapsed_s=elapsed)
    assert rc == fg21lib.FG21_E_DEVICE
    # only the first waiter's bit: the aborted warps stop without a bit of their own
    assert status == 1
    assert WAIT_LIMIT_S <= elapsed[0] < WAIT_LIMIT_S + 0.5
    for w in (1, 2, 3):
        # back through the abort signal, long before their own (8 s) limit
        assert elapsed[0] - 0.1 <= elapsed[w] <= elapsed[0] + 0.5
    assert "0x1" in fg21lib.lib().fg21_last_error().decode()

    # the context is still usable
    sky, obs, m, data = cases.small_case(npix=2048, N=5, F=31, T=7, window=3.0)
    model = fg21lib.fg21_build_regions(sky, obs, 5)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(129, 5, seed=11)
    got = fg21lib.fg21_loglike_batch(model, params, "fp16x3")
    want, _ = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance("fp16x3", m, obs, data, params)
    cases.check_logl("after_timeout_fp16x3", got, want, tol)
    assert fg21lib.fg21_model_sync_status(model) == 0
    model.close()
