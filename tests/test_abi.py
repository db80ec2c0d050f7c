"""The C-ABI boundary without a GPU: the library loads, exports every symbol
include/pilot.h declares, the binding mirrors them, and argument validation
that needs no device rejects bad inputs."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pilot.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pilot_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_21206_b300 import build
    build.build()
    from paper_2503_21206_b300 import pilot
    return pilot


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pilot_search" in names and "pilot_index_load" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(so, name), name


def test_binding_mirrors_the_header(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_defaults_and_version(lib):
    o = lib.pilot_search_options_default()
    assert (o.stage1, o.stage2_expansions, o.stage3, o.use_fes) == (1, 2, 1, 1)
    assert lib.pilot_abi_version() == 5


def _desc_arrays(n=8, d=4, dp=2, R=2):
    g = np.full((n, R), -1, np.int32)
    for i in range(n):
        g[i, 0] = (i + 1) % n
    mask = np.ones(n, np.uint8)
    return dict(graph=g, subgraph_mask=mask, subgraph=g.copy(), svd_basis=np.eye(d)[:, :dp].copy(),
                reduced_vecs=np.zeros((n, dp), np.float32), full_vecs=np.zeros((n, d), np.float32),
                entry_ids=np.array([0], np.int32))


@pytest.mark.parametrize("mutate, needle", [
    (lambda a: a["graph"].__setitem__((0, 1), 99), "outside"),
    (lambda a: a["graph"].__setitem__((0, 1), a["graph"][0, 0]), "repeats"),
    (lambda a: a["subgraph_mask"].__setitem__(1, 0), "unsampled"),
    (lambda a: a["full_vecs"].__setitem__((2, 1), np.nan), "non-finite"),
    (lambda a: a.__setitem__("entry_ids", np.array([9], np.int32)), "not a sampled"),
])
def test_load_rejects_malformed_index(lib, mutate, needle):
    a = _desc_arrays()
    mutate(a)
    with pytest.raises(lib.PilotError) as e:
        lib.pilot_index_load(**a)
    assert e.value.status == lib.PILOT_EINVAL
    assert needle in str(e.value)


def test_load_files_reports_io_and_format_errors(lib, tmp_path):
    with pytest.raises(lib.PilotError) as e:
        lib.pilot_index_load_files(str(tmp_path / "missing"))
    assert e.value.status == lib.PILOT_EIO
    (tmp_path / "pilot_index.txt").write_text("not an index\n")
    with pytest.raises(lib.PilotError) as e:
        lib.pilot_index_load_files(str(tmp_path))
    assert e.value.status == lib.PILOT_EFORMAT


def test_load_files_detects_corruption(lib, tmp_path, c1_small):
    from paper_2503_21206_b300 import index_build
    idx = c1_small[0]
    index_build.save_index(idx, str(tmp_path))
    raw = bytearray((tmp_path / "graph.bin").read_bytes())
    raw[100] ^= 0x40
    (tmp_path / "graph.bin").write_bytes(bytes(raw))
    with pytest.raises(lib.PilotError) as e:
        lib.pilot_index_load_files(str(tmp_path))
    assert e.value.status == lib.PILOT_EFORMAT and "checksum" in str(e.value)


def test_search_rejects_bad_arguments(lib):
    idx = lib.PilotIndex(0)
    q = np.zeros((1, 4), np.float32)
    with pytest.raises(lib.PilotError) as e:
        lib.pilot_search(idx, q, 1, 1)
    assert e.value.status == lib.PILOT_EINVAL
