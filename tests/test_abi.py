"""The C-ABI library builds, loads and exports every function include/nep.h declares;
host-side argument checks work without a GPU."""
import ctypes

import numpy as np
import os
import re

import pytest

from paper_2603_01234_gb300 import binding, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(nep_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for want in ("nep_create", "nep_destroy", "nep_compute", "nep_md_step", "nep_neighbors"):
        assert want in names
    assert set(names) == set(binding.EXPORTED)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version():
    binding.load(build_if_missing=True)
    lib = binding._lib
    assert lib.nep_error_string(0) == b"ok"
    assert lib.nep_error_string(-3) == b"neighbour list overflow"
    assert binding.nep_version() >= 1
    assert binding.nep_supported_shape(5, 4, 8, 8, 4)
    assert not binding.nep_supported_shape(3, 2, 5, 5, 4)
    # four-body l = 2 and five-body l = 1 terms, alone or together
    for l4, l5 in [(2, 0), (0, 1), (2, 1)]:
        assert binding.nep_supported_shape(5, 4, 8, 8, 4, l4, l5)
        assert binding.nep_supported_shape(5, 5, 9, 9, 4, l4, l5)
    for l4, l5 in [(1, 0), (3, 0), (0, 2), (4, 1)]:
        assert not binding.nep_supported_shape(5, 4, 8, 8, 4, l4, l5)


def test_create_rejects_bad_arguments_without_device():
    binding.load(build_if_missing=True)
    m = inputs.random_model(n_types=2, rc_radial=[[8.0, 7.0], [6.0, 8.0]], rc_angular=5.0)
    with pytest.raises(binding.NepError) as e:
        binding.nep_create(m)  # asymmetric cutoff table is rejected before any device call
    assert e.value.code == binding.NEP_ERR_ARG
    m = inputs.random_model(n_desc_radial=3)
    with pytest.raises(binding.NepError) as e:
        binding.nep_create(m)
    assert e.value.code == binding.NEP_ERR_UNSUPPORTED
    m = inputs.random_model(l_max_4b=1)  # the four-body term exists for l = 2 only
    with pytest.raises(binding.NepError) as e:
        binding.nep_create(m)
    assert e.value.code == binding.NEP_ERR_UNSUPPORTED
    m = inputs.random_model(l_max_4b=2)
    m.w0 = m.w0[:, :, :-1]  # w0 must hold N_des columns, four-body block included
    with pytest.raises(ValueError):
        binding.nep_create(m)


def test_virial_correction_closed_form():
    """Eq. 17: W -> W + (N_AA - N_CG) k_B T I (host function, no device)."""
    binding.load(build_if_missing=True)
    w = np.arange(9, dtype=np.float64)
    out = binding.nep_virial_correction(w, 1536, 512, 300.0)
    add = (1536 - 512) * 8.617333262e-5 * 300.0
    np.testing.assert_allclose(out, w + add * np.eye(3).reshape(9))
