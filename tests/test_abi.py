"""The C ABI without a GPU: libvio.so builds, loads and exports every
function include/vio.h declares; host-only calls validate their arguments."""
import ctypes
import os
import re

import pytest

from paper_2609_30459_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(vio_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    from paper_2609_30459_gb300 import vio
    return vio.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_2609_30459_gb300 import vio
    assert set(declared_functions()) <= set(vio.exported_symbols())


def test_params_default_follow_the_paper(lib):
    from paper_2609_30459_gb300 import vio
    p = vio.default_params()
    assert list(p.thresholds)[: p.n_thresholds] == [40, 20, 10, 5]
    assert p.k_per_cell == 1 and p.gn_iters == 5 and p.cell_w == p.cell_h == 50


def test_layout_geometry(lib):
    from paper_2609_30459_gb300 import vio
    L = vio.pyr_layout(1920, 1080, 5, 2048)
    assert list(L.w)[:5] == [1920, 960, 480, 240, 120]
    assert list(L.h)[:5] == [1080, 540, 270, 135, 67]
    assert L.pitch[0] == 2048
    for l in range(1, 5):
        assert L.pitch[l] % 128 == 0 and L.pitch[l] >= L.w[l]
        assert L.offset[l] % 256 == 0
        assert L.offset[l] + L.pitch[l] * L.h[l] <= L.upper_bytes
    assert L.upper_bytes % 256 == 0


def test_host_validation_rejects_bad_arguments(lib):
    from paper_2609_30459_gb300 import vio
    L = vio.PyrLayout()
    assert lib.vio_pyr_layout_make(0, 10, 2, 10, ctypes.byref(L)) == vio.ERR_INVALID_ARG
    assert lib.vio_pyr_layout_make(4, 4, 4, 4, ctypes.byref(L)) == vio.ERR_INVALID_ARG  # 0x0
    assert lib.vio_pyr_layout_make(10, 10, 9, 10, ctypes.byref(L)) == vio.ERR_INVALID_ARG
    assert lib.vio_pyr_layout_make(10, 10, 2, 9, ctypes.byref(L)) == vio.ERR_INVALID_ARG
    # null context / arguments are refused before anything touches the device
    assert lib.vio_pyramid_build(None, ctypes.byref(L), None, None) == vio.ERR_INVALID_ARG
    assert lib.vio_fast_scores(None, 10, 10, 10, None, None) == vio.ERR_INVALID_ARG
    assert lib.vio_fb_check(None, None, None, 1, 1, 0.2, None, None, None) == \
        vio.ERR_INVALID_ARG
    bad = vio.default_params(thresholds=(5, 10))          # increasing: refused
    h = ctypes.c_void_p()
    assert lib.vio_ctx_create(ctypes.byref(h), ctypes.byref(bad), 10, 10, 1) == \
        vio.ERR_INVALID_ARG
    assert lib.vio_frontend_step(None, None, 0, 0, None) == vio.ERR_INVALID_ARG
    assert lib.vio_status_string(vio.ERR_CUDA) == b"CUDA runtime error"


def test_product_has_no_cpu_fallback():
    # the binding must not reach for the oracle
    src = open(os.path.join(ROOT, "paper_2609_30459_gb300", "vio.py")).read()
    assert "oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_2609_30459_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2609_30459_gb300", "csrc",
                                                 f)).read().lower()


def test_host_validation_of_frontend_batch_and_server_calls(lib):
    """The frontend, batch, server and network entry points refuse null
    handles, misaligned buffers and out-of-range arguments on the host, before
    any device work."""
    from paper_2609_30459_gb300 import vio
    E = vio.ERR_INVALID_ARG
    buf = ctypes.create_string_buffer(64)
    # pipelined frontend calls: a null frontend
    assert lib.vio_frontend_run(None, buf, 16, 16, 32, 2, None) == E
    assert lib.vio_frontend_step_host_async(None, buf, buf, 16, 16, buf, buf, buf, buf, buf,
                                            None) == E
    # launch-shape tunes: a null handle
    good = vio.BatchTune(128, 0, 0, 0, 128, 0)
    assert lib.vio_frontend_set_tune(None, ctypes.byref(good)) == E
    assert lib.vio_batch_set_tune(None, ctypes.byref(good)) == E
    assert lib.vio_batch_get_tune(None, ctypes.byref(good)) == E
    # the network: null or misaligned buffers, a negative count
    assert lib.vio_initnet_forward(None, buf, 1, buf, None) == E
    addr = ctypes.addressof(buf)
    aligned = (addr + 15) & ~15
    assert lib.vio_initnet_forward(aligned, aligned + 2, 1, aligned, None) == E
    assert lib.vio_initnet_forward(aligned + 2, aligned, 1, aligned, None) == E
    assert lib.vio_initnet_forward(aligned, aligned, -1, aligned, None) == E
    # device-memory sizing and the server: null arguments, empty or oversized
    # class lists, requests out of time order
    b = ctypes.c_int64()
    assert lib.vio_batch_device_bytes(None, 1, ctypes.byref(b)) == E
    cls = vio._groups_array([(vio.default_params(n_levels=4, cell_w=32, cell_h=32), 640, 480,
                              2, 600)])
    assert lib.vio_batch_device_bytes(cls, 0, ctypes.byref(b)) == E
    assert lib.vio_batch_device_bytes(cls, 1, ctypes.byref(b)) == vio.OK and b.value > 0
    gap, over = ctypes.c_double(), ctypes.c_int64()
    assert lib.vio_server_loop_stats(None, ctypes.byref(gap), ctypes.byref(over)) == E
    reqs = (vio.ServerReq * 2)()
    done = (vio.ServerDone * 2)()
    n = ctypes.c_int64()
    assert lib.vio_server_run_trace(None, reqs, 2, done, 1.0, ctypes.byref(n)) == E
