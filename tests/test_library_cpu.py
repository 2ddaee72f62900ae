"""Host-side checks of the C ABI library that need no GPU: it builds, loads and
exports every entry point that include/hproj.h declares; the binding refuses
CPU tensors instead of falling back."""
import ctypes

import pytest

import paper_2109_09363_gb300 as hp
from paper_2109_09363_gb300 import build as hpbuild


@pytest.fixture(scope="module")
def lib():
    hpbuild.build()
    return hp.load_library()


def test_header_declares_the_boundary():
    names = hp.exported_symbols()
    for n in ["hp_ctx_create", "hp_ctx_destroy", "hp_face_mask", "hp_divergence",
              "hp_div_norms", "hp_project", "hp_jacobi_sweeps", "hp_status_string",
              "hp_advect_step", "hp_conv3x3_bf16", "hp_cnn_create", "hp_cnn_forward",
              "hp_project_hybrid", "hp_cnn_param_count",
              "hp_last_cuda_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in hp.exported_symbols():
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.hp_status_string(0) == b"ok"
    assert lib.hp_status_string(1) == b"invalid argument"


def test_argument_errors_are_returned_before_any_launch(lib):
    # null context / pointers are rejected on the host
    s = hp.hp_shape(1, 4, 4)
    prm = hp.hp_project_params(1e-3, 10, 0, 1.0, 1.0, 0, 1, 0)
    rc = lib.hp_project(None, None, None, None, s, ctypes.byref(prm), None, None, None, None,
                        None, None, None, 0, None)
    assert rc == 1
    assert lib.hp_face_mask(None, None, s, None) == 1
    assert lib.hp_divergence(None, None, None, None, hp.hp_shape(0, 4, 4), None) == 1


def test_binding_rejects_cpu_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(hp.HprojError):
        hp.hp_face_mask(torch.zeros((1, 4, 4), dtype=torch.uint8))


def test_cnn_parameter_count_matches_the_oracle(lib):
    from oracle import cnn as C
    assert int(lib.hp_cnn_param_count()) == C.param_count() == 372643
