"""The C ABI library loads and exports every symbol the public header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2310_10939_gb300 as fsc
from oracle import cluster as ocluster

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\*?\s*(fsc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(fsc.LIB_PATH):
        from paper_2310_10939_gb300 import build
        build.build()
    return fsc.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fsc_create_graph", "fsc_destroy_graph", "fsc_embed", "fsc_kmeans", "fsc_cluster",
                     "fsc_power_step", "fsc_default_params", "fsc_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    missing = []
    for name in declared_functions():
        try:
            getattr(L, name)
        except AttributeError:
            missing.append(name)
    assert not missing, missing


def test_host_only_calls(L):
    assert L.fsc_version().decode().count(".") == 2
    assert [fsc.pad_l(l) for l in range(0, 10)] == [0, 1, 2, 4, 4, 8, 8, 8, 8, 0]
    for n, k in [(1000, 4), (2 ** 20, 16), (154401, 8), (2 ** 22, 100), (500, 2), (50000, 20), (7, 1)]:
        assert fsc.default_params(n, k, 0) == ocluster.default_params(n, k)
        assert fsc.default_params(n, k, 1) == ocluster.paper_remark_params(n, k)
    with pytest.raises(fsc.FscError) as e:
        fsc.default_params(10, 11)
    assert e.value.name == "FSC_ERR_INVALID_ARG"
    for code in range(10):
        assert fsc.status_string(code) and fsc.status_string(code) != "unknown status"


def test_invalid_arguments_rejected_before_any_device_work(L):
    h = ctypes.c_void_p()
    assert L.fsc_create_graph(0, 0, None, None, None, 0, None, ctypes.byref(h)) == 1
    assert L.fsc_create_graph(5, 10, None, None, None, 0, None, ctypes.byref(h)) == 1
    assert L.fsc_embed(None, 2, 3, 0, 0, None, None, None) == 1
    assert L.fsc_kmeans(None, 10, 2, 2, 3, 0, 10, None, None, None, None, None) == 1
    assert L.fsc_cluster(None, 2, 2, 3, 0, 0, 10, None, None, None, None) == 1
