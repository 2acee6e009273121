"""The C ABI: the library builds for sm_103a, loads without a GPU, and exports
every entry point that include/nbody_gb300.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nbody_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1411_5234_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("nb_init", "nb_predict", "nb_force", "nb_correct", "nb_energy",
                     "nb_step_block"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_1411_5234_gb300 import nbody
    assert sorted(nbody.FUNCTIONS) == declared_functions()


def test_host_only_calls(libpath):
    # calls that never touch the device: config, sizes, error strings
    from paper_1411_5234_gb300 import nbody
    cfg = nbody.default_config()
    assert cfg.G == 1.0 and cfg.eta == 0.01 and cfg.precision == nbody.NB_MIXED
    assert nbody.workspace_size(1024, 1, cfg) > 1024 * 128
    assert nbody.workspace_size(2000, 7, cfg) >= nbody.workspace_size(1993, 1, cfg)
    with pytest.raises(nbody.NBError):
        nbody.workspace_size(0, 1, cfg)
    bad = nbody.default_config(level_min=5, level_max=3)
    with pytest.raises(nbody.NBError):
        nbody.workspace_size(100, 1, bad)
    assert nbody.strerror(nbody.NB_EINVAL) == "invalid argument"
    assert nbody.strerror(99) == "unknown status"


def test_missing_library_fails_loudly(tmp_path):
    import subprocess
    import sys
    env = dict(os.environ, NBODY_GB300_LIB=str(tmp_path / "nope.so"))
    r = subprocess.run([sys.executable, "-c", "import paper_1411_5234_gb300.nbody"], cwd=ROOT,
                       env=env, capture_output=True, text=True)
    assert r.returncode != 0 and "not found" in r.stderr


def test_precision_modes_in_config(libpath):
    from paper_1411_5234_gb300 import nbody
    for prec in (nbody.NB_FP64, nbody.NB_MIXED, nbody.NB_DS, nbody.NB_FP32):
        cfg = nbody.default_config(precision=prec)
        assert nbody.workspace_size(1000, 1, cfg) > 0
    with pytest.raises(nbody.NBError):
        nbody.workspace_size(1000, 1, nbody.default_config(precision=4))


def test_init_rejects_bad_workspaces_before_touching_the_device(libpath):
    """nb_init checks its arguments and the workspace size on the host and
    returns before any device call: too small a workspace is NB_ENOMEM (the
    library's analogue of an allocation failure: it allocates nothing
    itself), a misaligned one or bad particle data NB_EINVAL."""
    import ctypes
    import numpy as np
    from paper_1411_5234_gb300 import nbody
    lib = nbody.lib
    n = 64
    cfg = nbody.default_config()
    pos = np.zeros((n, 3)) + np.arange(n)[:, None]
    vel = np.zeros((n, 3))
    mass = np.full(n, 1.0 / n)
    off = np.array([0, n], dtype=np.int64)
    buf = np.zeros(1 << 16, dtype=np.uint8)
    base = buf.ctypes.data
    aligned = (base + 255) // 256 * 256
    need = nbody.workspace_size(n, 1, cfg)
    ctx = ctypes.c_void_p()

    def init(ptr, nbytes, m=mass, o=off):
        return lib.nb_init(ctypes.byref(ctx), ctypes.byref(cfg), 1, o.ctypes.data_as(ctypes.c_void_p),
                           m.ctypes.data_as(ctypes.c_void_p), pos.ctypes.data_as(ctypes.c_void_p),
                           vel.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(ptr), nbytes, None)

    assert need > 4096
    assert init(aligned, 4096) == nbody.NB_ENOMEM
    assert init(aligned + 8, need) == nbody.NB_EINVAL          # misaligned
    assert init(aligned, 4096, m=-mass) == nbody.NB_EINVAL     # negative masses
    bad_off = np.array([0, 0], dtype=np.int64)
    assert init(aligned, 4096, o=bad_off) == nbody.NB_EINVAL   # empty cluster
    assert not ctx.value


def test_workspace_memory_model(libpath):
    """~557 B per particle at large N in one workspace (both source layouts,
    partial sums, maps): N = 2^20 fits in 0.6 GB, 280 GB hold ~5e8."""
    from paper_1411_5234_gb300 import nbody
    cfg = nbody.default_config()
    per = [nbody.workspace_size(n, 1, cfg) / n for n in (1 << 20, 1 << 24)]
    assert all(500 < p < 620 for p in per), per
    assert nbody.workspace_size(1 << 20, 1, cfg) < 0.6e9
    # many small clusters cost a little more per particle (per-cluster tiles)
    assert nbody.workspace_size(2007990, 512, cfg) / 2007990 < 620
