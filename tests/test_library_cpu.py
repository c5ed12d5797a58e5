"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point include/steps.h declares; the binding marshals."""
import os
import re

import numpy as np
import pytest

from paper_1811_05903_gb300 import build as libbuild
from paper_1811_05903_gb300 import steps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(steps_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return steps.load()


def test_header_parses():
    names = declared_functions()
    assert "steps_init" in names and "steps_forces" in names and "steps_kdk_step" in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    assert sorted(steps.HEADER_SYMBOLS) == [n for n in declared_functions() if n in steps.HEADER_SYMBOLS]
    assert set(declared_functions()) <= set(steps.HEADER_SYMBOLS) | {n for n in declared_functions()
                                                                     if n not in steps.HEADER_SYMBOLS}


def test_host_only_entry_points(lib):
    cfg = steps.steps_default_config()
    assert cfg.G == 1.0 and cfg.prec == steps.STEPS_F32_COMP and cfg.mode == steps.STEPS_STATIC
    assert lib.steps_strerror(steps.STEPS_ETIMEOUT) == b"device-side wait timed out"
    names = steps.steps_variants()
    assert len(names) == lib.steps_num_variants() and all(names)
    assert lib.steps_variant_name(-1) is None


def test_argument_validation_without_gpu(lib):
    # rejected on the host before any CUDA call
    with pytest.raises(steps.StepsError) as e:
        steps.steps_init(np.zeros((0, 3)), None, np.zeros(0))
    assert e.value.status == steps.STEPS_EINVAL
    cfg = steps.make_config(prec=7)
    with pytest.raises(steps.StepsError) as e:
        steps.steps_init(np.zeros((2, 3)), None, np.ones(2), cfg=cfg)
    assert e.value.status == steps.STEPS_EINVAL
    assert lib.steps_forces(None, None) == steps.STEPS_EINVAL
    assert lib.steps_kdk_step(None, 0.1, None) == steps.STEPS_EINVAL
    assert lib.steps_size(None) == 0
    lib.steps_free(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(steps, "_lib", None)
    monkeypatch.setattr(libbuild, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(OSError):
        steps.load()


def test_emulator_validation_without_gpu(lib):
    p = np.zeros(steps.STEPS_EMU_NPARAMS, np.float32)
    with pytest.raises(steps.StepsError) as e:
        steps.Emulator(p, batch=100)  # not a multiple of 64: rejected before any CUDA call
    assert e.value.status == steps.STEPS_EINVAL
    p[3] = np.inf
    with pytest.raises(steps.StepsError) as e:
        steps.Emulator(p, batch=64)
    assert e.value.status == steps.STEPS_EINVAL
