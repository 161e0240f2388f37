"""The C ABI library without a GPU: it loads, exports every function that
include/sgf.h declares, and rejects malformed descriptors on the host before
any device work (no compute call is made here)."""
import re
from pathlib import Path

import pytest

import __graft_entry__
from paper_1603_03142_gb300 import workloads as W

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_1603_03142_gb300 import sgf
    return sgf


def declared_functions():
    text = (ROOT / "include" / "sgf.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgf_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib._lib, name), name
    assert sorted(lib.EXPORTS) == names


def test_version(lib):
    assert "sm_103a" in lib.version()


@pytest.mark.parametrize("bad", [
    dict(n=13), dict(n=6), dict(n=0), dict(levels=0), dict(levels=9), dict(n=16, levels=5),
    dict(off=[(0, 0), (9, 0)]), dict(off=[(0, 0), (-1, 0)]), dict(h0=-1.0),
])
def test_invalid_descriptors_rejected_on_host(lib, bad):
    args = dict(n=16, levels=2, off=[(0, 0), (4, 4)], h0=0.125)
    args.update(bad)
    nest = W.Nest(n=max(args["n"], 1), levels=max(args["levels"], 1), h0=args["h0"], off=args["off"])
    nest.n = args["n"]
    nest.levels = args["levels"]
    if args["levels"] > len(nest.off):
        nest.off = nest.off + [(0, 0)] * (args["levels"] - len(nest.off))
    assert lib.create_status(nest, "fp32") == lib.SGF_EINVAL
    assert "n" in lib.last_error() or "level" in lib.last_error() or "off" in lib.last_error() or "h0" in lib.last_error()


def test_unsupported_sizes_rejected_on_host(lib):
    assert lib.create_status(W.Nest(n=8192), "fp32") == lib.SGF_EUNSUPPORTED
    assert lib.create_status(W.Nest(n=4096), "fp64") == lib.SGF_EUNSUPPORTED


def test_unknown_precision(lib):
    assert lib.create_status(W.Nest(n=16), 7) == lib.SGF_EINVAL


def test_zero_rim_flag_rules(lib):
    # SGF_PLAN_ZERO_RIM is a single-level option; unknown flags are rejected
    assert lib.create_status(W.Nest(n=16, levels=2, off=[(0, 0), (4, 4)]), "fp32", lib.PLAN_ZERO_RIM) == lib.SGF_EINVAL
    assert lib.create_status(W.Nest(n=16), "fp32", 0x80) == lib.SGF_EINVAL
