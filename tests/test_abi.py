"""The C ABI on a machine without a GPU: the library loads, exports every
symbol include/fg21.h declares, and its host-side paths (argument checks,
region building, data simulation) behave; compute calls fail loudly."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2603_13196_gb300 import fg21, inputs as I

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fg21.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fg21_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    return fg21.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    names = set(declared_functions())
    assert names <= set(fg21._SIGS), names - set(fg21._SIGS)


def test_version_and_device_count(L):
    assert fg21.fg21_version().startswith("fg21")
    assert fg21.fg21_device_count() >= 0


def test_argument_errors_without_device(L):
    nul = C.c_void_p(None)
    assert L.fg21_loglike_batch(nul, nul, 1, nul, 0, nul) == fg21.FG21_E_ARG
    assert L.fg21_loglike_batch_device(nul, nul, 1, nul, 0, nul) == fg21.FG21_E_ARG
    assert L.fg21_model_set_data(nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_model_info(nul, nul, nul, nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_serve_create(nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_serve_wait(nul, 1, 0) == fg21.FG21_E_ARG
    assert L.fg21_model_destroy(nul) == fg21.FG21_OK
    assert L.fg21_serve_destroy(nul) == fg21.FG21_OK
    assert L.fg21_graph_create_multi(nul, nul, nul, nul, 1, 0, nul) == fg21.FG21_E_ARG
    assert L.fg21_graph_launch(nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_graph_sync_status(nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_graph_destroy(nul) == fg21.FG21_OK
    assert L.fg21_model_shape(nul, nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_build_regions_ab(nul, nul, nul, nul, nul, nul, nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_build_regions_ab_host(nul, nul, nul, nul, nul, nul, nul, nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_selftest_bounded_wait(nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_selftest_mma_rounding(nul, nul, nul, nul, nul) == fg21.FG21_E_ARG
    assert L.fg21_model_sync_status(nul, nul, nul) == fg21.FG21_E_ARG
    assert "NULL" in L.fg21_last_error().decode()


def test_build_regions_rejects_bad_inputs(L):
    sky = I.make_sky(256, 1)
    obs = I.make_obs(5, 2, 1.0)
    with pytest.raises(fg21.Fg21Error) as e:
        fg21.fg21_build_regions_host(sky, obs, 0)
    assert e.value.code == fg21.FG21_E_ARG
    with pytest.raises(fg21.Fg21Error):
        fg21.fg21_build_regions_host(sky, obs, 300)          # N > npix
    bad = I.Sky(dirs=sky.dirs * 1.1, t230=sky.t230, beta=sky.beta)
    with pytest.raises(fg21.Fg21Error):
        fg21.fg21_build_regions_host(bad, obs, 3)            # not unit vectors
    nanb = I.Sky(dirs=sky.dirs, t230=sky.t230, beta=np.where(np.arange(256) == 3, np.nan, sky.beta))
    with pytest.raises(fg21.Fg21Error):
        fg21.fg21_build_regions_host(nanb, obs, 3)
    with pytest.raises(KeyError):
        fg21.fg21_build_regions_host(sky, obs, 3, scheme="nope")


def test_compute_calls_fail_loudly_without_device(L):
    if fg21.fg21_device_count() > 0:
        pytest.skip("a GPU is present")
    sky = I.make_sky(256, 1)
    obs = I.make_obs(5, 2, 1.0)
    with pytest.raises(fg21.Fg21Error) as e:
        fg21.fg21_build_regions(sky, obs, 3)
    assert e.value.code == fg21.FG21_E_CUDA
    o = fg21.fg21_serve_opts(1 << 30, 4096, 100, 2, 0, 0)
    h = C.c_void_p()
    assert L.fg21_serve_create(C.byref(o), C.byref(h)) == fg21.FG21_E_CUDA
