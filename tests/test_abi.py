"""The C-ABI library builds, loads and exports every symbol include/pald.h
declares; host-side argument checks reject bad calls without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2307_16652_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "pald.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pald_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("pald_focus", "pald_cohesion", "pald_batched", "pald_host", "pald_validate",
                 "pald_status_string", "pald_release"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in pald.h but not exported"


def test_status_strings_and_version(lib):
    for s in range(9):
        assert isinstance(binding.pald_status_string(s), str) and binding.pald_status_string(s)
    assert binding.pald_version() >= 100
    assert binding.pald_schedule_count() >= 1
    assert binding.pald_schedule_name(0)
    assert binding.pald_schedule_name(99) is None


def test_invalid_arguments_are_rejected_on_the_host(lib):
    o = binding.PaldOpts(0, 0, -1, 0)
    INVALID = 1
    fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert lib.pald_focus(None, 8, fake, ctypes.byref(o), None) == INVALID
    assert lib.pald_focus(fake, 1, fake, ctypes.byref(o), None) == INVALID        # n < 2
    assert lib.pald_focus(fake, 1 << 21, fake, ctypes.byref(o), None) == INVALID  # n too large
    assert lib.pald_cohesion(fake, None, 8, fake, ctypes.byref(o), None) == INVALID
    bad = binding.PaldOpts(0, 7, -1, 0)                                           # unknown accum mode
    assert lib.pald_cohesion(fake, fake, 8, fake, ctypes.byref(bad), None) == INVALID
    bad = binding.PaldOpts(0, 0, -1, 2)                                           # unknown flag bit
    assert lib.pald_focus(fake, 8, fake, ctypes.byref(bad), None) == INVALID
    assert lib.pald_validate(None, 8, None) == INVALID
    assert lib.pald_host(None, 8, None, None, None) == INVALID
    assert lib.pald_tie_map(None, 8, fake, None) == INVALID
    assert lib.pald_tie_map(fake, 1, fake, None) == INVALID
    assert lib.pald_local_depth(None, 8, fake, None) == INVALID
    assert lib.pald_cohesion_depth(fake, fake, 8, fake, None, ctypes.byref(o), None) == INVALID  # null L
    assert lib.pald_cohesion_depth(fake, fake, 1, fake, fake, ctypes.byref(o), None) == INVALID
    assert lib.pald_local_depth(fake, 1, fake, None) == INVALID
    assert lib.pald_strong_ties(fake, 8, float("nan"), fake, None) == INVALID
    assert lib.pald_strong_ties(fake, 8, 0.5, None, None) == INVALID


def test_tie_map_size():
    # nb = ceil(n/64) blocks, wpp = ceil(ceil(n/G)/32) words per block pair, plus nb dirty words;
    # groups of G = 8 y up to n = 65536, 32 y beyond
    assert binding.pald_tie_map_words(1) == 0
    assert binding.pald_tie_map_words(2) == 1 * 1 * 1 + 1
    assert binding.pald_tie_map_words(64) == 1 + 1
    assert binding.pald_tie_map_words(65) == 2 * 2 * 1 + 2
    assert binding.pald_tie_map_words(256) == 4 * 4 * 1 + 4
    assert binding.pald_tie_map_words(257) == 5 * 5 * 2 + 5
    assert binding.pald_tie_map_words(1024) == 16 * 16 * 4 + 16
    assert binding.pald_tie_map_words(1025) == 17 * 17 * 5 + 17
    assert binding.pald_tie_map_words(65536) == 1024 * 1024 * 256 + 1024
    assert binding.pald_tie_map_words(65537) == 1025 * 1025 * 65 + 1025
    assert binding.pald_tie_map_words(147456) == 2304 * 2304 * 144 + 2304


def test_batched_argument_checks(lib):
    o = binding.PaldOpts(0, 0, -1, 0)
    fake = ctypes.c_void_p(256)

    def call(ns, offs):
        ns = np.asarray(ns, dtype=np.int64)
        offs = np.asarray(offs, dtype=np.int64)
        return lib.pald_batched(len(ns), ns.ctypes.data, offs.ctypes.data, fake, fake, fake, ctypes.byref(o), None)

    assert call([32, 40], [0, 1024 + 1]) == 1     # misaligned offset
    assert call([32, 40], [0, 1000]) == 1         # overlaps the first matrix (32*32 = 1024)
    assert call([1, 40], [0, 1024]) == 1          # n < 2
    assert call([5000], [0]) == 1                 # n beyond the batched limit
    assert lib.pald_batched(0, None, None, fake, fake, fake, ctypes.byref(o), None) == 1


def test_binding_refuses_cpu_tensors(lib):
    torch = pytest.importorskip("torch")
    D = torch.zeros(4, 4)
    U = torch.zeros(4, 4, dtype=torch.int32)
    with pytest.raises(ValueError):
        binding.pald_focus(D, U)
