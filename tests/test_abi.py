"""CPU-only checks of the C ABI library: it builds, loads without a GPU, exports every entry
point include/vol.h declares, and its pure-host layout planner follows the chunking rules."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import _capi
    return _capi


def declared():
    text = open(os.path.join(ROOT, "include", "vol.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vol_[a-z_]+)\s*\(", text)) - {"vol_provider_fn"})


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 18
    assert sorted(lib.EXPORTS) == names
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n


def test_every_declaration_cites_its_passage():
    """Each entry point's comment in vol.h names the passage of the paper it follows (a section
    or figure), or says that the paper has no counterpart."""
    text = open(os.path.join(ROOT, "include", "vol.h")).read()
    cite = re.compile(r"Sec\. (III|IV|V|VI)-?[A-H]?|Fig\. \d|no counterpart|[Nn]ot in the paper")
    missing = []
    for m in re.finditer(r"^(?:int|void|const char \*)\s*(vol_[a-z_]+)\s*\(", text, flags=re.M):
        # the comment block directly above the declaration (#define lines in between belong to it)
        lines = text[:m.start()].rstrip().split("\n")
        while lines and lines[-1].startswith("#define"):
            lines.pop()
        before = "\n".join(lines)
        if not before.endswith("*/"):
            missing.append(m.group(1))
            continue
        block = re.sub(r"\s*\n\s*\*?\s*", " ", before[before.rfind("/*"):])
        if not cite.search(block):
            missing.append(m.group(1))
    assert not missing, f"declarations without a passage: {missing}"
    assert len(re.findall(r"^(?:int|void|const char \*)\s*vol_", text, flags=re.M)) >= 20


def test_struct_sizes_match_header(lib):
    # sizes follow from the field lists in vol.h (natural alignment)
    assert ctypes.sizeof(lib.vol_camera) == 4 * 14 + 8
    assert ctypes.sizeof(lib.vol_params) == 4 * 2 + 16 + 4 * 9
    assert ctypes.sizeof(lib.vol_trace_rec) == 56


def test_plan_chunk_addressing(lib):
    from paper_2509_26213_gb300.volume import plan
    lay = plan((1000, 7, 1), "u16", 16, 4)
    assert [tuple(lay.level_dims[l]) for l in range(4)] == [(1000, 7, 1), (500, 4, 1), (250, 2, 1), (125, 1, 1)]
    assert [tuple(lay.level_bricks[l]) for l in range(4)] == [(63, 1, 1), (32, 1, 1), (16, 1, 1), (8, 1, 1)]
    assert list(lay.level_pt_offset[:4]) == [0, 63, 95, 111]
    assert lay.total_bricks == 119
    assert lay.slot_bytes == ((4 * 16 * 16 * 17 * 2 + 255) // 256) * 256   # quad: B*B*(B+1) entries of 4
    assert lay.nslots == 119
    cmp = plan((1000, 7, 1), "u16", 16, 4, layout="compact")
    assert cmp.slot_bytes == ((17 ** 3 * 2 + 255) // 256) * 256         # compact: (B+1)^3 voxels
    assert (lay.layout, lay.entry_voxels, cmp.layout, cmp.entry_voxels) == (0, 4, 1, 1)
    c3 = plan((2048, 2048, 2048), "u8", 32, 6)
    assert c3.total_bricks == 64 ** 3 + 32 ** 3 + 16 ** 3 + 8 ** 3 + 4 ** 3 + 2 ** 3
    # a cache budget caps the slot count
    c5 = plan((4096, 4096, 4096), "u8", 64, 7, cache_bytes=16 << 30)
    assert c5.nslots == (16 << 30) // c5.slot_bytes


@pytest.mark.parametrize("bad", [dict(brick=24), dict(brick=2), dict(levels=0), dict(levels=17),
                                 dict(dims=(0, 4, 4)), dict(dtype=9)])
def test_plan_rejects(lib, bad):
    args = dict(dims=(64, 64, 64), dtype=0, brick=16, levels=2)
    args.update(bad)
    lay = lib.vol_layout()
    d = (ctypes.c_int64 * 3)(*args["dims"])
    rc = lib.load().vol_plan(d, args["dtype"], args["brick"], args["levels"], 0, 0, ctypes.byref(lay))
    assert rc == lib.VOL_ERR_INVALID_ARG


def zettabyte_figures():
    """The figures Sec. V-C prints for its virtual volume (tests/golden/zettabyte_volume.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "zettabyte_volume.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_plan_sparse_page_table(lib):
    """The paper's virtual 2 ZB volume (8,000,000^3 voxels, 128^3 bricks): too many bricks for a
    flat table, a few hundred MB of top grids for the sparse one."""
    from paper_2509_26213_gb300.volume import plan
    z = zettabyte_figures()
    n, B = int(z["voxels_per_axis"]), int(z["brick_edge"])
    # the printed size: 8,000,000^3 voxels at 4 bytes is 2 ZB, and its 62,500^3 bricks fit the
    # printed three-level tree of 2^16-entry pages (2^48 leaves) -- "the upper limit"
    assert abs(n ** 3 * z["bytes_per_voxel"] / z["total_bytes_order"] - 1) < 0.03
    assert (n // B) ** 3 <= int(z["page_table_entries_per_page"]) ** int(z["page_table_levels"]) < 2 * (n // B) ** 3
    D = (n,) * 3
    with pytest.raises(RuntimeError):
        plan(D, "f32", B, 8, cache_bytes=16 << 30)
    with pytest.raises(RuntimeError):  # a sparse table needs a cache budget
        plan(D, "f32", B, 8, sparse_pt=True)
    lay = plan(D, "f32", B, 8, cache_bytes=16 << 30, sparse_pt=True)
    assert lay.sparse_pt == 1
    assert lay.level_bricks[0][0] == n // B == 62500 and lay.total_bricks > 2 ** 47
    tops = [(-(-lay.level_bricks[l][0] // 256)) ** 3 for l in range(8)]
    assert list(lay.level_pt_offset[:8]) == [sum(tops[:l]) for l in range(8)]
    assert lay.pt_top_entries == sum(tops) and lay.pt_top_entries * 4 < (1 << 30)
    assert lay.nslots == (16 << 30) // lay.slot_bytes


def test_plan_the_benchmark_volumes(lib):
    """The printed sizes of the Table I volumes follow from their printed dimensions and types,
    and both plan as out-of-core volumes of 64^3 bricks with a 16 GiB cache (flat page tables)."""
    import os
    from paper_2509_26213_gb300.volume import plan
    path = os.path.join(os.path.dirname(__file__), "golden", "benchmark_volumes.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    bpv = {"u16": 2, "f32": 4}
    for name, x, y, z, dtype, gb, mode in rows:
        D = (int(x), int(y), int(z))
        size = D[0] * D[1] * D[2] * bpv[dtype]
        assert abs(size / 1e9 - float(gb)) < 1.0, (name, size)
        lay = plan(D, dtype, 64, 8, cache_bytes=16 << 30)
        assert tuple(lay.level_bricks[0][a] for a in range(3)) == tuple(-(-d // 64) for d in D)
        assert lay.nslots == (16 << 30) // lay.slot_bytes and lay.sparse_pt == 0
        assert mode in ("dvr", "mop")


def test_missing_library_fails_loudly(lib, monkeypatch, tmp_path):
    import importlib
    from paper_2509_26213_gb300 import _capi
    monkeypatch.setattr(_capi, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(_capi, "_lib", None)
    with pytest.raises(ImportError):
        _capi.load()
