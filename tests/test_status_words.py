"""The status words that the decode and topology kernels raise on the device map to the status
and message sim_set_population returns (include/voxsim.h, sim_check_status_words).  The words are
injected on the host: no test makes a device-side wait run out."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    return voxsim


def check(vs, words):
    w = np.asarray(words, dtype=np.int32)
    st = vs.lib().sim_check_status_words(w.ctypes.data_as(C.c_void_p))
    return st, vs.lib().sim_last_error(None).decode()


def test_mlp_wait_gave_up_maps_to_timeout(lib):
    st, msg = check(lib, [0, 4, 0, 0])
    assert st == lib.SIM_ETIMEOUT and "MLP" in msg and "gave up" in msg


def test_labelling_bound_maps_to_timeout(lib):
    st, msg = check(lib, [1, 0, 0, 0])
    assert st == lib.SIM_ETIMEOUT and "labelling" in msg


def test_bad_material_maps_to_einval(lib):
    st, msg = check(lib, [2, 0, 0, 0])
    assert st == lib.SIM_EINVAL and "material" in msg


def test_timeout_wins_over_other_flags_and_clear_words_pass(lib):
    assert check(lib, [3, 4, 0, 0])[0] == lib.SIM_ETIMEOUT
    assert check(lib, [0, 0, 0, 0])[0] == lib.SIM_OK
    assert check(lib, [0, 1, 0, 0])[0] == lib.SIM_OK      # bits no kernel raises are ignored


def test_null_words_rejected(lib):
    assert lib.lib().sim_check_status_words(None) == lib.SIM_EINVAL


def test_lattice_segment_wait_gave_up_maps_to_timeout(lib):
    st, msg = check(lib, [0, 0, 8, 0])
    assert st == lib.SIM_ETIMEOUT and "segment" in msg and "gave up" in msg
