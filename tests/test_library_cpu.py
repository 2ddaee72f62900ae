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
    prm = hp.hp_project_params(1e-3, 10, 0, 1.0, 1.0, 0, 1, 0, 0, 0, 0)
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
    assert int(lib.hp_cnn_arch_param_count(0)) == C.param_count("multiscale")
    assert int(lib.hp_cnn_arch_param_count(1)) == C.param_count("smallscale") == 123491
    assert hp.CNN.param_count("smallscale") == 123491
    assert int(lib.hp_cnn_arch_param_count(2)) == C.param_count("monoscale") == 222497
    assert int(lib.hp_cnn_arch_param_count(3)) == C.param_count("unet") == 388545
    assert int(lib.hp_cnn_arch_param_count(4)) == -1
    assert int(lib.hp_cnn_arch_param_count(-1)) == -1


def test_cnn_architecture_argument_checks(lib):
    out = hp._P()
    # unknown architecture, bad shape, null handle: rejected before any device call
    assert lib.hp_cnn_create_arch(ctypes.byref(out), 5, hp.hp_shape(1, 64, 64), 0) == 1
    assert not out
    assert lib.hp_cnn_create_arch(ctypes.byref(out), 1, hp.hp_shape(1, 62, 64), 0) == 1
    assert lib.hp_cnn_create_arch(None, 1, hp.hp_shape(1, 64, 64), 0) == 1
    # the Unet's five scales need sizes that are multiples of 16
    assert lib.hp_cnn_create_arch(ctypes.byref(out), 3, hp.hp_shape(1, 40, 48), 0) == 1
    assert lib.hp_cnn_get_arch(None) == -1
    with pytest.raises(ValueError):
        hp.CNN.param_count("resnet")


def test_ctypes_structures_match_the_header(tmp_path):
    """The binding's structures have the sizes and field offsets the C compiler
    gives the header's (the ABI the Python names marshal into)."""
    import os
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "hproj.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu\\n", sizeof(hp_shape), sizeof(hp_project_params),\n'
        "         sizeof(hp_plume_params), sizeof(hp_train_params));\n"
        '  printf("%zu %zu %zu %zu %zu\\n", offsetof(hp_plume_params, scheme),\n'
        "         offsetof(hp_project_params, fixed_iters), offsetof(hp_train_params, lambda_div),\n"
        "         offsetof(hp_project_params, inflow_x1), offsetof(hp_plume_params, open_top));\n"
        "  return 0; }\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    sizes = [int(x) for x in out[:4]]
    offs = [int(x) for x in out[4:]]
    assert sizes == [ctypes.sizeof(hp.hp_shape), ctypes.sizeof(hp.hp_project_params),
                     ctypes.sizeof(hp.hp_plume_params), ctypes.sizeof(hp.hp_train_params)]
    assert offs == [hp.hp_plume_params.scheme.offset, hp.hp_project_params.fixed_iters.offset,
                    hp.hp_train_params.lambda_div.offset, hp.hp_project_params.inflow_x1.offset,
                    hp.hp_plume_params.open_top.offset]


def test_architecture_numbers_match_the_header(tmp_path):
    """The binding's architecture names map to the header's hp_cnn_arch values,
    and the initial parameters of every architecture have the oracle's size."""
    import os
    import subprocess
    from oracle import cnn as C
    from paper_2109_09363_gb300 import training as T
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "arch.c"
    src.write_text(
        '#include <stdio.h>\n#include "hproj.h"\n'
        "int main(void) {\n"
        '  printf("%d %d %d %d\\n", HP_CNN_MULTISCALE, HP_CNN_SMALLSCALE, HP_CNN_MONOSCALE,\n'
        "         HP_CNN_UNET);\n"
        "  return 0; }\n")
    exe = tmp_path / "arch"
    r = subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [hp.CNN_ARCHS[a] for a in ("multiscale", "smallscale", "monoscale", "unet")]
    for arch in hp.CNN_ARCHS:
        n = C.param_count(arch)
        assert hp.CNN.param_count(arch) == n
        assert T.init_params(seed=0, arch=arch).size == n


def test_new_entry_points_reject_null_arguments(lib):
    s = hp.hp_shape(1, 4, 4)
    assert lib.hp_plume_head(None, s, 1.0, 0.01, None, None) == 1
    assert lib.hp_cnn_check(None) == 1
    assert lib.hp_trainer_pdnn_gradient(None, None, None, None, s, 1, None, None, None) == 1
    assert lib.hp_status_string(7) == b"a tensor-core wait timed out"
    pp = hp.PlumeParams(scheme=1).c()
    assert lib.hp_advect_step(None, None, None, None, None, None, None, s, ctypes.byref(pp),
                              None) == 1


def test_paper_plume_geometry():
    import numpy as np
    from paper_2109_09363_gb300 import workloads as W
    n = 512
    fl, (x0, x1) = W.paper_plume_geometry(n)
    assert x1 - x0 == round(0.29 * n) and (x0 + x1) / 2 == n / 2
    # disc of diameter 0.312 n, centre 0.625 n above the bottom wall
    r, cy = 0.156 * n, n - 0.625 * n
    assert fl[int(cy), n // 2] == 1 and fl.sum() == pytest.approx(np.pi * r * r, rel=0.01)
    rows = np.nonzero(fl.any(axis=1))[0]
    assert (rows.min() + rows.max() + 1) / 2 == pytest.approx(cy, abs=1.0)
    fl0, _ = W.paper_plume_geometry(n, cylinder=False)
    assert fl0.sum() == 0


def test_shapes_beyond_the_launch_limits_are_rejected_on_the_host(lib):
    # batch and ny each map to one CUDA grid dimension (65535 blocks); larger
    # shapes return HP_ERR_INVALID_ARG before any CUDA call, so stand-in
    # pointers that are never dereferenced suffice here
    fake = ctypes.c_void_p(256)
    for shape in [(1, 70000, 1), (70000, 1, 1), (1, 65535, 4), (65535, 4, 4)]:
        s = hp.hp_shape(*shape)
        assert lib.hp_divergence(fake, fake, fake, fake, s, None) == 1
        assert lib.hp_face_mask(fake, fake, s, None) == 1
        assert lib.hp_div_norms_noalloc(fake, fake, fake, fake, fake, s, None) == 1
        pp = hp.PlumeParams().c()
        assert lib.hp_advect_step(fake, fake, fake, fake, fake, fake, fake, s,
                                  ctypes.byref(pp), None) == 1


def _checkpoint_bytes(arch, n, step=0, moments=False, seed=0):
    """A checkpoint in the layout include/hproj.h documents, written here."""
    import struct
    import numpy as np
    rng = np.random.default_rng(seed)
    body = struct.pack("<8sIiqqII", b"HPCNNCK1", 1, arch, n, step, int(moments), 0)
    body += rng.standard_normal(n).astype("<f4").tobytes()
    if moments:
        body += rng.standard_normal(2 * n).astype("<f4").tobytes()
    h = 1469598103934665603
    for byte in body:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return body + struct.pack("<Q", h)


def test_checkpoint_reader_errors_need_no_gpu(lib, tmp_path):
    import struct
    out = ctypes.c_void_p()
    s = hp.hp_shape(1, 64, 64)
    assert lib.hp_cnn_load(ctypes.byref(out), str(tmp_path / "missing").encode(), s, 0) == 8
    assert not out.value
    assert lib.hp_cnn_load(None, b"x", s, 0) == 1
    assert lib.hp_trainer_load(None, b"x") == 1
    assert lib.hp_status_string(8) == b"checkpoint file error"
    n = int(lib.hp_cnn_arch_param_count(1))
    good = _checkpoint_bytes(1, n)
    for bad in (good[:-1], good[:50], good + b"\0",
                good[:60] + bytes([good[60] ^ 4]) + good[61:],      # a parameter bit
                _checkpoint_bytes(1, n - 1),                        # wrong count
                _checkpoint_bytes(7, n),                            # unknown arch
                # a header announcing 2^31 parameters in a file of a few
                # bytes: rejected on the file size, before any allocation
                struct.pack("<8sIiqqII", b"HPCNNCK1", 1, 1, 2 ** 31, 0, 0, 0) + bytes(64)):
        p = tmp_path / "bad.hpcnn"
        p.write_bytes(bad)
        assert lib.hp_cnn_load(ctypes.byref(out), str(p).encode(), s, 0) == 8
        assert not out.value
    # the documented layout passes the reader: creating the network is the
    # first step that needs a GPU (HP_ERR_CUDA here, without one)
    p = tmp_path / "good.hpcnn"
    p.write_bytes(good)
    rc = lib.hp_cnn_load(ctypes.byref(out), str(p).encode(), s, 0)
    torch = pytest.importorskip("torch")
    assert rc == (0 if torch.cuda.is_available() else 2)
    if rc == 0:
        lib.hp_cnn_destroy(out)
