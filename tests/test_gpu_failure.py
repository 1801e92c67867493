"""Failure paths on the GPU without a GPU fault: the device's bounded wait (the guard on every tile copy)
run out on a barrier that nothing completes, and the host watchdog on a stream wait run out by a tiny
limit. Both return HYDRO_ETIMEOUT and leave the context usable; nothing hangs or traps. Also the
arithmetic-peak probe that cross-checks the ALU roofline."""
import os
import time

import numpy as np
import pytest

from paper_1507_08549_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _hydro():
    from paper_1507_08549_gb300 import hydro
    return hydro


def test_device_wait_runs_out_and_the_context_stays_usable():
    hydro = _hydro()
    prob = wl.advected_wave(64)
    h = hydro.Hydro(prob, dtype="f64")
    try:
        t0 = time.perf_counter()
        rc = h.wait_selftest(1 << 16)
        assert rc == hydro.ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        assert b"device wait" in h.lib.hydro_last_error(h.ctx)
        # the next call works and gives the same bits as a fresh context
        U = h.state(prob.U0)
        h.step(U, 5)
        h2 = hydro.Hydro(prob, dtype="f64")
        V = h2.state(prob.U0)
        h2.step(V, 5)
        assert np.array_equal(U.cpu().numpy(), V.cpu().numpy())
        h2.close()
        with pytest.raises(hydro.HydroError):
            h._check(h.lib.hydro_wait_selftest(h.ctx, 0), "polls 0")
    finally:
        h.close()


def test_host_watchdog_times_out_and_recovers():
    import torch
    hydro = _hydro()
    prob = wl.blobs_blast(2048)
    h = hydro.Hydro(prob, dtype="f32")
    U = h.state(prob.U0)
    ref = h.state(prob.U0)
    old = os.environ.get("HYDRO_TIMEOUT_S")
    try:
        os.environ["HYDRO_TIMEOUT_S"] = "1e-6"
        with pytest.raises(hydro.HydroError) as e:
            h.step(U, 20)  # ~20 ms of work against a 1 microsecond limit
        assert e.value.code == hydro.ETIMEOUT
    finally:
        if old is None:
            del os.environ["HYDRO_TIMEOUT_S"]
        else:
            os.environ["HYDRO_TIMEOUT_S"] = old
    torch.cuda.synchronize()  # the work itself was never stopped: it completes
    h.step(ref, 20)
    assert np.array_equal(U.cpu().numpy(), ref.cpu().numpy())
    h.step(U, 1)  # and the context keeps working
    h.close()


def test_fma_probe_measures_the_arithmetic_peaks():
    """The measured FMA rates that cross-check the arithmetic roofline: FP32 within 20 % of 152 SMs x 128
    lanes x clock (no more than that), FP64 far below FP32 on this part."""
    import torch
    hydro = _hydro()
    prob = wl.advected_wave(32)
    h = hydro.Hydro(prob, dtype="f32")
    try:
        f32 = h.fma_probe("f32", 16384)
        f64 = h.fma_probe("f64", 256)
    finally:
        h.close()
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2.2e9  # above the maximum SM clock
    assert 0.5 * derived < f32 <= derived
    assert 0 < f64 < 0.1 * f32
    with pytest.raises(hydro.HydroError):
        h2 = hydro.Hydro(prob, dtype="f32")
        try:
            h2.fma_probe("f32", 0)
        finally:
            h2.close()
