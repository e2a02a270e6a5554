"""The C-ABI library builds, loads and exports every entry point of include/tdb.h
(no GPU needed: nothing here calls into the device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(tdb_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1912_03174_gb300 import binding
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1912_03174_gb300 import binding
    assert sorted(binding.SIGNATURES) == _declared()


def test_status_strings_and_defaults(lib):
    from paper_1912_03174_gb300 import binding as B
    assert B.tdb_status_string(0) == "ok"
    assert "unstable" in B.tdb_status_string(6)
    p = B.tdb_default_params()
    assert p.dt == 0.2 and p.scc == 1 and p.precision == 0 and p.history_cap == 65536


def test_workspace_size_is_host_only_and_validates(lib):
    from paper_1912_03174_gb300 import binding as B
    from paper_1912_03174_gb300 import inputs as I
    s, run = I.flake_c2()
    p = B.make_params(run, "fp64")
    nb = B.tdb_workspace_bytes(s, p)
    N = s.n_orb
    assert nb > 11 * N * N * 8          # S, S^-1, H0, 4 rho levels, X re/im, M, H
    assert nb < 16 * N * N * 8
    p32 = B.make_params(run, "fp32")
    assert B.tdb_workspace_bytes(s, p32) > nb
    bad = B.make_params(run, "fp64")
    bad.dt = 0.0
    assert B.tdb_workspace_bytes(s, bad) == 0


def test_missing_library_fails_loudly(tmp_path):
    from paper_1912_03174_gb300 import binding
    with pytest.raises(RuntimeError):
        binding.load(str(tmp_path / "nope.so"))


def test_without_a_device_calls_fail_with_a_status(lib):
    # on a host with no usable GPU the library returns TDB_ERR_CUDA with a message
    # (no abort, no CPU fallback); on a GPU host there is nothing to check here
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1912_03174_gb300 import binding as B
    from paper_1912_03174_gb300 import inputs as I
    sysm, run = I.chain_c1()
    with pytest.raises(B.TdbError) as e:
        B.tdb_create(sysm, B.make_params(run, "fp64"))
    assert e.value.status == 3 and "CUDA device" in str(e.value)   # TDB_ERR_CUDA
    with pytest.raises(B.TdbError) as e:
        B.ShiftNet(8, 16)
    assert e.value.status == 3
