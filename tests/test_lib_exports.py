"""CPU checks of the C ABI: the library builds, loads and exports every
function include/apc.h declares (no compute calls: there is no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(apc_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1708_01413_gb300 import apc, build
    build.build()
    L = apc.lib()
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(L, name), name
    assert set(apc.EXPORTED) <= set(declared)


def test_optimal_params_host_entry_matches_oracle():
    # apc_optimal_params is pure host arithmetic: callable without a GPU
    from oracle import apc_oracle as O
    from paper_1708_01413_gb300 import apc
    for lo, hi in ((1e-4, 0.9), (0.3, 0.31), (5e-8, 1.0)):
        g, e, r = apc.apc_optimal_params(lo, hi)
        g0, e0, r0 = O.optimal_params(lo, hi)
        assert g == pytest.approx(g0, rel=1e-12) and e == pytest.approx(e0, rel=1e-12)
        assert r == pytest.approx(r0, rel=1e-12)
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_optimal_params(0.5, 0.2)
    assert ei.value.name == "INVALID_ARG"


def test_product_path_has_no_oracle_import():
    # the product package never imports the oracle
    pkg = os.path.join(ROOT, "paper_1708_01413_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from\s+oracle|import\s+oracle)", text, flags=re.M), f


def test_hb_optimal_params_host_entry_matches_oracle():
    # pure host arithmetic: Sec. 6 preconditioning makes the Hessian m X
    from oracle import apc_oracle as O
    from paper_1708_01413_gb300 import apc
    for lo, hi, m in ((1e-4, 0.9, 8), (0.3, 0.31, 3), (5e-8, 1.0, 128)):
        a, b, r = apc.apc_hb_optimal_params(lo, hi, m)
        a0, b0, r0 = O.hb_optimal_params(m * lo, m * hi)
        assert a == pytest.approx(a0, rel=1e-12) and b == pytest.approx(b0, rel=1e-12)
        assert r == pytest.approx(r0, rel=1e-12)
        assert r == pytest.approx(O.optimal_params(lo, hi)[2], rel=1e-9)  # the APC rate
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_hb_optimal_params(0.5, 0.2, 4)
    assert ei.value.name == "INVALID_ARG"


def test_tile_cache_key_and_store(tmp_path):
    # the tuner's cache: power-of-two histograms of n and p, k and the SM
    # count make the key; a stored choice is read back, other keys miss
    from paper_1708_01413_gb300 import apc
    k1 = apc.tile_cache_key([300, 310, 4000], [16, 20, 128], 32, 152)
    assert k1 == apc.tile_cache_key([4000, 310, 300], [128, 16, 20], 32, 152)  # order does not matter
    assert k1 != apc.tile_cache_key([300, 310, 4000], [16, 20, 128], 16, 152)
    assert k1 != apc.tile_cache_key([300, 310, 4000], [16, 20, 128], 32, 148)
    assert k1 != apc.tile_cache_key([300, 600, 4000], [16, 20, 128], 32, 152)
    path = str(tmp_path / "tiles.json")
    assert apc.load_tiles(k1, path) is None
    apc.store_tiles(k1, (128, 256, 1, 2, 2, 4), path)
    apc.store_tiles("other", (256, 512, 2, 0, 1, 1), path)
    assert apc.load_tiles(k1, path) == (128, 256, 1, 2, 2, 4)
    assert apc.load_tiles("missing", path) is None
