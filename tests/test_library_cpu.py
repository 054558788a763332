"""CPU checks of the C-ABI library: it builds, loads, exports every entry point declared in
include/he.h, and its host-side sampler table equals the oracle's (no GPU calls)."""
import ctypes
import os
import re

import pytest

from oracle import prng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libhe():
    from paper_2102_03494_gb300 import build_ext, he
    build_ext.build()
    return he


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "he.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|uint64_t|const char\*)\s+(he_[a-z0-9_]+)\(", text, re.M)))


def test_library_exports_every_declared_symbol(libhe):
    lib = ctypes.CDLL(libhe.LIB_PATH)
    names = declared_entry_points()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(libhe.exported_symbols())


def test_sampler_table_matches_oracle(libhe):
    assert libhe.he_gaussian_table() == prng.cdt_table()


def test_binding_refuses_to_run_without_gpu(libhe):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        libhe.Context(log_n=10, n_q=2, n_p=1, alpha=1)


def header_constants():
    """Every NAME = value inside the header's enums and its #define'd int32 constants."""
    text = open(os.path.join(ROOT, "include", "he.h")).read()
    out = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", text):
        for name, val in re.findall(r"(HE_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            out[name] = int(val)
    for name, val in re.findall(r"#define\s+(HE_[A-Z0-9_]+)\s+\(\(int32_t\)(0x[0-9a-fA-F]+)\)", text):
        v = int(val, 16)
        out[name] = v - (1 << 32) if v >= 1 << 31 else v
    return out


def test_binding_constants_match_the_header(libhe):
    consts = header_constants()
    assert {"HE_OK", "HE_ETIMEOUT", "HE_NTT", "HE_DP_DP", "HE_ROW_SWAP", "HE_RELIN_KEY"} <= set(consts)
    for name, val in consts.items():
        if name.startswith("HE_PHASE_") or name == "HE_N_PHASES":
            continue
        assert getattr(libhe, name) == val, name
    # phase indices: the binding's names follow the header's order
    phases = sorted((v, n) for n, v in consts.items() if n.startswith("HE_PHASE_"))
    assert [n[len("HE_PHASE_"):].lower() for _, n in phases] == list(libhe.Context.PHASES[:len(phases)])


def test_binding_declares_a_signature_for_every_entry_point(libhe):
    assert set(libhe._SIGS) == set(declared_entry_points())
