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
    assert [fsc.pad_l(l) for l in range(0, 10)] == [0, 1, 2, 4, 4, 8, 8, 8, 8, 16]
    assert [fsc.pad_l(l) for l in (16, 17, 32, 33, 64, 65, 100, 128, 129)] == [16, 32, 32, 64, 64, 128, 128, 128, 0]
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
    rp = (ctypes.c_int64 * 6)()
    assert L.fsc_create_graph(5, 0, rp, None, None, 0x8, None, ctypes.byref(h)) == 1   # unknown flag
    assert L.fsc_embed(None, 2, 3, 0, 0, None, None, None) == 1
    assert L.fsc_kmeans(None, 10, 2, 2, 3, 0, 10, None, None, None, None, None) == 1
    assert L.fsc_cluster(None, 2, 2, 3, 0, 0, 10, None, None, None, None) == 1


EXAMPLE = os.path.join(ROOT, "paper_2310_10939_gb300", "examples", "cluster_cliques.c")


def _cuda_home():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return d
    return None


def build_c_example(out_path, source=None):
    """Compile the C example (or another C program) against include/fsc.h and link it with
    libfsc.so (plain C, gcc)."""
    import shutil
    import subprocess
    cuda = _cuda_home()
    if shutil.which("gcc") is None or cuda is None:
        pytest.skip("gcc or the CUDA toolkit headers are not available")
    if not os.path.exists(fsc.LIB_PATH):
        from paper_2310_10939_gb300 import build
        build.build()
    lib_dir = os.path.dirname(fsc.LIB_PATH)
    cudalib = next((os.path.join(cuda, d) for d in ("lib64", "lib", "targets/sbsa-linux/lib",
                                                    "targets/x86_64-linux/lib")
                    if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), os.path.join(cuda, "lib64"))
    cmd = ["gcc", "-O2", "-Wall", "-Wextra", "-Werror", "-std=c99", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(cuda, "include"), source or EXAMPLE, "-L" + lib_dir, "-lfsc", "-L" + cudalib, "-lcudart",
           "-Wl,-rpath," + lib_dir, "-Wl,-rpath," + cudalib, "-o", str(out_path)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return out_path


def test_c_example_builds_against_the_header(tmp_path):
    """The boundary is usable from C alone: the example compiles warning-free and links."""
    assert os.path.exists(build_c_example(tmp_path / "cluster_cliques"))


@pytest.mark.gpu
def test_c_example_recovers_disjoint_cliques(tmp_path):
    """Run the C example: 8 disjoint 64-cliques come out as 8 clusters (Sec. 2: the components
    span the top eigenspace of M)."""
    import subprocess
    exe = build_c_example(tmp_path / "cluster_cliques")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "cliques recovered: yes" in r.stdout


def test_binding_flags_match_the_header():
    """The Python binding's flag constants are the header's."""
    import re
    text = open(os.path.join(ROOT, "include", "fsc.h")).read()
    defs = {m.group(1): int(m.group(2), 16) for m in re.finditer(r"#define FSC_(\w+)\s+0x([0-9a-fA-F]+)u", text)}
    for name in ("VALIDATE_SYMMETRY", "COPY", "EMBED_RESCALE", "BATCH_AUTOTUNE", "FILTER_NO_FALLBACK"):
        assert defs[name] == getattr(fsc, name), name


RESET = os.path.join(ROOT, "tests", "c", "reset_cycles.c")


def test_reset_cycles_program_builds(tmp_path):
    assert os.path.exists(build_c_example(tmp_path / "reset_cycles", RESET))


@pytest.mark.gpu
def test_library_state_survives_device_reset(tmp_path):
    """Three create / embed / k-means / cluster / destroy cycles with cudaDeviceReset between them
    (a C program, so that no other runtime state outlives the reset): the library rebuilds its
    memory pool, status word and launch attributes in each new context."""
    import subprocess
    exe = build_c_example(tmp_path / "reset_cycles", RESET)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=180)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("cliques recovered") == 3
