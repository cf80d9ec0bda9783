"""Host-side checks of libgf2x_gb300.so: it loads, exports every symbol the
header declares, and its plan algebra reproduces the paper's sizes.  No GPU."""
import json
import os
import re

import pytest

from paper_2201_10473_gb300 import build as pbuild
from paper_2201_10473_gb300 import gf2x

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CONFIG_SIZES = [12323, 17669, 24659, 35851, 40973, 57637]


@pytest.fixture(scope="module", autouse=True)
def built():
    pbuild.build()


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(gf2x_[a-z0-9_]+)\s*\(", text,
                                re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 15
    L = gf2x.lib()
    for name in names:
        assert hasattr(L, name), name


def test_experiment_libraries_load_and_export_their_test_entries():
    import ctypes

    from paper_2201_10473_gb300 import build
    build.build()
    tc = ctypes.CDLL(build.experiment_lib("libgf2x_exp_tc.so"))
    assert hasattr(tc, "gf2x_exp_tc_mul512") and hasattr(tc, "gf2x_exp_comb_mul512")
    bs = ctypes.CDLL(build.experiment_lib("libgf2x_exp_bitsliced.so"))
    assert hasattr(bs, "gf2x_exp_bitsliced_leaves")
    bs.gf2x_exp_bitsliced_group.restype = ctypes.c_int
    assert [bs.gf2x_exp_bitsliced_group(m) for m in range(4)] == [7, 4, 8, 0]


def test_binding_flags_match_the_header():
    text = open(os.path.join(ROOT, "include", "gf2x_gb300.h")).read()
    defines = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define GF2X_([A-Z_]+)\s+\(?([0-9x]+)u", text)}
    for name in ("REDUCE", "BATCH_PERSISTENT", "BATCH_ITEMS_ON_DEVICE", "BATCH_LARGEST_FIRST", "BATCH_SHARED_A",
                 "BATCH_DYNAMIC"):
        assert getattr(gf2x, name) == defines[name], name
    assert gf2x.HOST_INPUTS_READY == 1 << 8 and "HOST_INPUTS_READY" in text
    batch = [v for k, v in defines.items() if k.startswith("BATCH_")]
    assert len(set(batch)) == len(batch) and all(v & (v - 1) == 0 for v in batch)   # distinct single bits


def test_entries_reject_a_null_context_without_a_gpu():
    L = gf2x.lib()
    assert L.gf2x_mul_unbalanced(None, None, None, 100, 2, None, 50, 1, 1, 3, None) == 1
    assert L.gf2x_mulmod_sparse(None, None, None, None, 3, 100, 1, 2, 3, 2, None) == 1
    assert L.gf2x_mul_toom4(None, None, None, None, 100, 1, 2, 4, 0, None) == 1
    assert L.gf2x_mul_toom5(None, None, None, None, 100, 1, 2, 4, 0, None) == 1
    assert L.gf2x_mul_strided(None, None, None, None, 100, 1, 2, 4, 0, gf2x.BATCH_SHARED_A, None) == 1
    assert L.gf2x_sparse_info_get(100, None) == 1


def _prototypes():
    text = open(os.path.join(ROOT, "include", "gf2x_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for ret, name, params in re.findall(r"\b(gf2x_status|const char \*|void|uint32_t)\s*(gf2x_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                                        text):
        yield ret, name, [p.strip() for p in params.split(",")]


def test_every_context_entry_rejects_a_null_context_without_a_gpu():
    """Every entry point whose first argument is a context returns
    GF2X_EINVAL for a null one before it touches any other argument or the
    GPU (the header's error rule); destroy(NULL) is a no-op."""
    import ctypes
    L = gf2x.lib()
    checked = 0
    for ret, name, params in _prototypes():
        if params[0] != "gf2x_ctx *ctx":
            continue
        fn = getattr(L, name)
        if ret == "gf2x_status":
            types = getattr(fn, "argtypes", None) or [None] * len(params)
            args = [None if t is None or issubclass(t, (ctypes.c_void_p, ctypes.c_char_p, ctypes._Pointer)) else 0
                    for t in types]
            assert fn(*args) == 1, name     # restype as the binding declared it (an int status)
            checked += 1
        elif ret == "void":
            fn.restype = None
            fn(None)
        else:
            fn.restype = ctypes.c_char_p
            assert fn(None)
    assert checked >= 20


def test_status_strings_and_version():
    L = gf2x.lib()
    assert L.gf2x_status_str(0) == b"ok"
    assert b"sm_103a" in L.gf2x_version()
    for s in range(8):
        assert L.gf2x_status_str(s)


def _chains(elem):
    """Karatsuba chains (leaf S, levels) whose top size is exactly `elem` words."""
    for S in (16, 12, 10, 8, 6, 4):
        if elem % S:
            continue
        r = elem // S
        for lead in (1, 3, 5):
            if r % lead:
                continue
            r2 = r // lead
            if r2 & (r2 - 1) == 0:
                yield S, ([f"K{lead}"] if lead > 1 else []) + ["K2"] * (r2.bit_length() - 1)


def test_paper_sizes_through_the_abi():
    """The library's planner reproduces every printed size (Sec. 3.2 size rule)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_plan_sizes.json")))
    checked = 0
    for case in g["cases"]:
        n = case["bits"]
        if len(case["levels"]) > 1 or n > 80000:
            continue  # two Toom levels, or too large for one CTA: sizes checked in test_plan_algebra
        elem = case["elem_bits"] // 32
        info = None
        for S, chain in _chains(elem):
            if len(chain) + 1 > gf2x.MAX_LEVELS:
                continue
            for seq in (0, 1):
                try:
                    info = gf2x.plan_info(n, ".".join(case["levels"] + chain) + f"/{S}/0/{seq}")
                    break
                except gf2x.Gf2xError:
                    pass
            if info:
                break
        assert info is not None, case
        assert 32 * info["top_words"] == case["bits"], (case, info)
        assert info["level_words"][1] == elem
        checked += 1
    assert checked >= 13


@pytest.mark.parametrize("n", CONFIG_SIZES + [1, 2, 63, 64, 65, 1000, 4096, 65536, 100000, 120001, 131072])
def test_default_plan_covers_n_and_fits(n):
    spec = gf2x.default_spec(n)
    info = gf2x.plan_info(n, spec)
    assert 32 * info["top_words"] >= n
    assert info["smem_bytes"] <= 232448
    assert info["threads"] % 32 == 0 and 128 <= info["threads"] <= 1024
    assert info["ops_leaf"] <= info["ops_full"]


def test_clmul_counts_table_compkarat_through_abi():
    for r in range(1, 6):
        t = 2 ** r
        for lead, mult in ((None, 1), (3, 6), (5, 15)):
            chain = ([f"K{lead}"] if lead else []) + ["K2"] * r
            spec = ".".join(chain) + "/4"
            words = 4 * (lead or 1) * t
            info = gf2x.plan_info(32 * words, spec)
            # 4-word leaves are 2x2 64-bit schoolbooks: 4 clmul64 each
            assert info["clmul64"] == 4 * mult * 3 ** r


def test_spec_parse_roundtrip_and_errors():
    s = gf2x.parse_spec("T2.K3.K2.K2/8/288/0/1/1")
    assert gf2x.spec_text(s) == "T2.K3.K2.K2/8/288/0/1/1"
    assert gf2x.spec_text(gf2x.parse_spec("K3")) == "K3/0/0/0/0/0"
    for bad in ["K4/8", "X2", "T0", "K2/7", "K2/8/100", "K2/8/0/1", "K2/8/0/0/9", "K3/8/0/0/1", "K2/12/0/0/1",
                "K2/8/0/0/0/2", "K2/8/0/0/0/1", "K2/8/0/0/0/0/0"]:
        with pytest.raises(gf2x.Gf2xError):
            gf2x.parse_spec(bad)


def test_plan_rejections():
    with pytest.raises(gf2x.Gf2xError) as e:
        gf2x.plan_info(17669, "K2/8")           # does not cover n
    assert e.value.status == 5
    with pytest.raises(gf2x.Gf2xError):
        gf2x.plan_info(0, "K2/8")
    with pytest.raises(gf2x.Gf2xError):
        gf2x.plan_info(131073, "K2/8")
    with pytest.raises(gf2x.Gf2xError):
        gf2x.plan_info(57637, "K5.K3.K2.K2.K2/16/0/0")  # breadth-first does not fit shared memory


def test_seq_top_reduces_shared_memory():
    with pytest.raises(gf2x.Gf2xError):
        gf2x.plan_info(57637, "T16.K5.K2.K2.K2.K2/8/0/0")   # breadth first: too much shared memory
    seq = gf2x.plan_info(57637, "T16.K5.K2.K2.K2.K2/8/0/1")
    assert seq["smem_bytes"] <= 232448
    assert 32 * seq["top_words"] == 58368


def test_paper_hqc_plans_through_the_abi():
    """The HQC multiplication timing table of Sec. 4: hqc-128 at 18048 bits (Toom3Karat3, w=64) and hqc-256 at
    58368 bits (Toom3Karat5, w=512)."""
    a = gf2x.plan_info(17669, "T2.K3.K2.K2.K2/8")
    assert 32 * a["top_words"] == 18048 and a["nleaves"] == 5 * 6 * 27
    b = gf2x.plan_info(57637, "T16.K5.K2.K2.K2.K2/8/0/1")
    assert 32 * b["top_words"] == 58368 and b["nleaves"] == 5 * 15 * 81


def test_split_plan_facts():
    """Split plans: the top level's children are products of E0 words; the
    size rule is the same; scratch is nch x 2E0 words per product."""
    info = gf2x.plan_info(57637, "T16.K5.K2.K2.K2.K2/8/0/0/1/1")
    assert 32 * info["top_words"] == 58368
    assert info["level_words"][:2] == [1824, 640]
    assert info["scratch_bytes"] == 4 * 5 * 2 * 640
    assert info["nleaves"] == 5 * 15 * 81          # leaf products (the fused level counted at its leaves)
    whole = gf2x.plan_info(57637, "T16.K5.K2.K2.K2.K2/8/0/1/1/0")
    assert whole["nleaves"] == info["nleaves"]
    assert gf2x.plan_info(131072, None)["scratch_bytes"] > 0      # only split plans reach the maximum size


def test_packaged_plan_database_and_logs_are_consistent():
    """Every database entry is a valid plan for its size and is the fastest
    record of its (size, bucket) in the shipped timing logs -- of the
    one-CTA-per-product log where that log covers the bucket, else of the
    persistent-launch logs; the single-product plans chosen for the plain
    baselines are one-launch plans."""
    import gzip
    import json

    from paper_2201_10473_gb300 import autotune
    db = autotune.load_db(gf2x.PACKAGED_PLAN_DB)
    recs = autotune.packaged_log()
    with gzip.open(autotune.PACKAGED_SINGLE_LOG, "rt") as f:
        recs += [json.loads(line) for line in f if line.strip()]
    cta = autotune.packaged_cta_log()
    assert cta and all(r["launch"] == "cta" for r in cta)
    assert len(db) >= 24
    for (n, bucket), e in db.items():
        info = gf2x.plan_info(n, e["spec"])
        assert 32 * info["top_words"] >= n
        same = [r for r in cta if r["n"] == n and autotune.batch_bucket(r["batch"]) == bucket]
        if not same:
            same = [r for r in recs if r["n"] == n and autotune.batch_bucket(r["batch"]) == bucket]
        assert same, (n, bucket)
        assert min(same, key=lambda r: r["ms"])["spec"] == e["spec"], (n, bucket)
    single = autotune.single_product_plans([12323, 17669, 24659, 35851, 40973, 57637])
    assert len(single) == 6 and all(not s.endswith("/1") for s in single.values())
