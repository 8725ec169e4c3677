"""Host-side checks of librmat that need no GPU: the library loads, exports
every function that include/rmat.h declares, validates arguments, and builds
tables identical (field by field) to the oracle's independent construction."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300 import _capi, build as rm_build
from paper_1905_03525_gb300.workloads import G500, SKEWED, noisy_levels

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ASYM = (0.5, 0.2, 0.25, 0.05)


@pytest.fixture(scope="module", autouse=True)
def built():
    rm_build.build()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(rmat_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rmat_build_table", "rmat_generate", "rmat_free_table", "rmat_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(_capi.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    bound = {name for name, _, _ in _capi.SIGNATURES}
    assert set(declared_functions()) <= bound


def _compare(lib_export, ot):
    N = 1 << ot.bits
    assert lib_export["entries"] == ot.entries
    assert lib_export["bits"] == ot.bits
    assert lib_export["max_len"] == ot.max_len
    for f in ("sym", "len", "p", "w", "thr", "alias"):
        a, b = lib_export[f], getattr(ot, f)
        assert a.shape == (N,)
        assert np.array_equal(a, b), f


@pytest.mark.parametrize("params,k,bound", [
    (G500, 26, 4096), (G500, 16, 256), (ASYM, 20, 1000), (SKEWED, 30, 8192), (SKEWED, 64, 5000),
    (G500, 4, 4096), (G500, 30, 5), (G500, 34, 1 << 16), ((0.25, 0.25, 0.25, 0.25), 20, 4096),
    ((0.6, 0.2, 0.2, 0.0), 12, 777)])
def test_variable_table_matches_oracle(params, k, bound):
    t = rm.rmat_build_table(*params, k, bound)
    _compare(rm.rmat_table_export(t), oracle.Table.variable(*params, k, bound))


@pytest.mark.parametrize("params,ell", [(G500, 4), (ASYM, 1), (ASYM, 6), (SKEWED, 9), ((1.0, 0, 0, 0), 3)])
def test_fixed_table_matches_oracle(params, ell):
    t = rm.rmat_build_table_fixed(*params, 20, ell)
    _compare(rm.rmat_table_export(t), oracle.Table.fixed([params], ell))


@pytest.mark.parametrize("k,ell", [(34, 6), (34, 5), (7, 3), (12, 12), (64, 4)])
def test_level_tables_match_oracle(k, ell):
    P = noisy_levels(k, seed=k * 100 + ell)
    t = rm.rmat_build_table_levels(P, k, ell)
    groups = oracle.level_groups(P, k, ell)
    info = rm.rmat_table_info(t)
    assert info["groups"] == len(groups)
    for g, ot in enumerate(groups):
        _compare(rm.rmat_table_export(t, g), ot)


def test_table_info():
    t = rm.rmat_build_table(*G500, 26, 4096)
    info = rm.rmat_table_info(t)
    assert info["entries"] == 4093 and info["bits"] == 12 and info["index_bytes"] == 4
    assert info["max_len"] == 13 and info["groups"] == 1
    assert info["device_image_bytes"] == 4096 * 12 + 4 * 64 * 4
    t64 = rm.rmat_build_table_levels(noisy_levels(34), 34, 6, rm.RMAT_UNDIRECTED)
    i64 = rm.rmat_table_info(t64)
    assert i64["index_bytes"] == 8 and i64["groups"] == 6 and i64["flags"] == 1


@pytest.mark.parametrize("call", [
    lambda: rm.rmat_build_table(0.5, 0.5, 0.5, 0.5, 10, 4096),
    lambda: rm.rmat_build_table(*G500, 0, 4096),
    lambda: rm.rmat_build_table(*G500, 65, 4096),
    lambda: rm.rmat_build_table(*G500, 10, 4),
    lambda: rm.rmat_build_table(*G500, 10, (1 << 24) + 1),
    lambda: rm.rmat_build_table(float("nan"), 0.2, 0.2, 0.6, 10, 100),
    lambda: rm.rmat_build_table(-0.1, 0.5, 0.5, 0.1, 10, 100),
    lambda: rm.rmat_build_table_fixed(*G500, 10, 0),
    lambda: rm.rmat_build_table_fixed(*G500, 10, 13),
    lambda: rm.rmat_build_table_levels(np.tile(G500, (10, 1)), 10, 0),
    lambda: rm.rmat_build_table_levels(np.tile(G500, (65, 1)), 65, 1),
    lambda: rm.rmat_build_table_levels(np.tile(G500, (10, 1)), 10, 2, flags=8),
])
def test_invalid_arguments_are_rejected_on_host(call):
    with pytest.raises(rm.RmatError) as ei:
        call()
    assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    assert ei.value.message


def test_generate_argument_checks_need_no_device():
    t = rm.rmat_build_table(*G500, 26, 4096)
    with pytest.raises(rm.RmatError) as ei:
        rm.rmat_generate(t, 1, 0, 10, 0)          # NULL output
    assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    with pytest.raises(rm.RmatError) as ei:
        rm.rmat_generate(t, 1, 0, 10, 0x1004)     # misaligned
    assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    with pytest.raises(rm.RmatError) as ei:
        rm.rmat_generate(t, 1, 2 ** 64 - 5, 10, 0x1000)  # index overflow
    assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    rm.rmat_generate(t, 1, 0, 0, 0)               # count == 0 is a no-op


MAX_EDGES = 1 << 56   # RMAT_MAX_EDGES of include/rmat.h


def test_counts_near_2p64_are_rejected_on_host():
    """Counts whose ceiling divisions by a tile or a work unit would wrap
    (2^64 - 1 edges from offset 0) stop at the per-call maximum, before any
    device work; the maximum itself passes the host checks."""
    t = rm.rmat_build_table(*G500, 26, 4096)
    for count in ((1 << 64) - 1, (1 << 64) - 512, MAX_EDGES + 1):
        with pytest.raises(rm.RmatError) as ei:
            rm.rmat_generate(t, 1, 0, count, 0x1000)
        assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT and "RMAT_MAX_EDGES" in ei.value.message
        with pytest.raises(rm.RmatError) as ei:
            rm.rmat_generate_host(t, 1, 0, count, 0x1000)
        assert "RMAT_MAX_EDGES" in ei.value.message
        with pytest.raises(rm.RmatError) as ei:
            rm.rmat_generate_naive(G500, 26, 0, 1, 0, count, 0x1000)
        assert "RMAT_MAX_EDGES" in ei.value.message
        b = rm.rmat_batch_create()
        with pytest.raises(rm.RmatError) as ei:
            rm.rmat_batch_add(b, t, 1, 0, count, 0x1000)
        assert "RMAT_MAX_EDGES" in ei.value.message
        with pytest.raises(rm.RmatError) as ei:
            rm.rmat_partition_create(t, 2, count, 1)
        assert "RMAT_MAX_EDGES" in ei.value.message
        with pytest.raises(rm.RmatError) as ei:
            rm.rmat_generate_batch_noalloc([t], [1], [0], [count], [0x1000])
        assert "RMAT_MAX_EDGES" in ei.value.message
    b = rm.rmat_batch_create()
    rm.rmat_batch_add(b, t, 1, 0, MAX_EDGES, 0x1000)
    assert rm.rmat_batch_size(b) == (1, MAX_EDGES)


def test_batch_host_checks():
    b = rm.rmat_batch_create()
    t = rm.rmat_build_table(*G500, 20, 1000)
    rm.rmat_batch_add(b, t, 1, 0, 100, 0x1000)
    rm.rmat_batch_add(b, t, 2, 5, 200, 0x2000)
    assert rm.rmat_batch_size(b) == (2, 300)
    with pytest.raises(rm.RmatError):
        rm.rmat_batch_add(b, t, 1, 0, 10, 0x1004)
    with pytest.raises(rm.RmatError):
        rm.rmat_batch_add(b, t, 1, 2 ** 64 - 1, 10, 0x1000)
    b.free()


def test_launch_config_roundtrip_and_checks():
    t = rm.rmat_build_table(*G500, 26, 4096)
    rm.rmat_set_launch_config(t, 256, 4, 128)
    assert rm.rmat_get_launch_config(t) == {"threads": 256, "ctas_per_sm": 4, "tile_edges": 128}
    with pytest.raises(rm.RmatError):
        rm.rmat_set_launch_config(t, 100, 1, 128)
    with pytest.raises(rm.RmatError):
        rm.rmat_set_launch_config(t, 256, 1, 40)


def test_server_create_fails_cleanly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_1905_03525_gb300.serve import Server
    with pytest.raises(rm.RmatError):
        Server(1 << 30)


@pytest.mark.parametrize("kind,params,k,t,m,seed,rows", [
    ("variable", G500, 26, 5, 1 << 30, 1, None),
    ("variable", SKEWED, 30, 8, 1 << 34, 7, (37, 200)),
    ("fixed", ASYM, 16, 4, 1 << 20, 3, (5, 6)),
    ("variable", G500, 20, 0, 12345, 9, None),
    ("variable", ASYM, 12, 12, 3000, 2, (100, 4096)),
    ("variable", G500, 40, 10, 1 << 40, 11, (0, 3)),
    ("variable", (0.25, 0.25, 0.25, 0.25), 24, 6, 999_999, 5, None),
    ("fixed", (1.0, 0.0, 0.0, 0.0), 10, 3, 777, 1, None),
])
def test_partition_tiles_match_oracle(kind, params, k, t, m, seed, rows):
    """The library's host-side divide and conquer (its own Philox and
    binomials) gives the oracle's tiles, counts and edge numbers exactly."""
    table = rm.rmat_build_table(*params, k, 4096) if kind == "variable" else rm.rmat_build_table_fixed(*params, k, 4)
    r0, r1 = rows if rows else (0, 1 << t)
    p = rm.rmat_partition_create(table, t, m, seed, r0, r1)
    got = rm.rmat_partition_tiles(p)
    ref = oracle.partition(params, t, m, seed, r0, r1)
    for f in ("row", "col", "count", "first"):
        assert np.array_equal(got[f], ref[f]), f
    assert rm.rmat_partition_info(p) == (len(ref["row"]), int(ref["count"].sum()))


def test_partition_host_checks():
    t = rm.rmat_build_table(*G500, 20, 1024)
    for args in [(21, 100, 1, 0, 1 << 21), (5, 100, 1, 3, 2), (5, 100, 1, 0, 33), (-1, 100, 1, 0, 1)]:
        with pytest.raises(rm.RmatError):
            rm.rmat_partition_create(t, *args)
    lv = rm.rmat_build_table_levels(noisy_levels(20), 20, 5)
    with pytest.raises(rm.RmatError):
        rm.rmat_partition_create(lv, 3, 100, 1)
    u = rm.rmat_build_table(*G500, 20, 1024)
    rm.rmat_table_set_flags(u, rm.RMAT_UNDIRECTED)
    with pytest.raises(rm.RmatError):
        rm.rmat_partition_create(u, 3, 100, 1)
    b = rm.rmat_batch_create()
    with pytest.raises(rm.RmatError):
        rm.rmat_batch_add_tile(b, t, 1, 0, 10, 4, 16, 0, 8)    # tile row >= 2^4
    with pytest.raises(rm.RmatError):
        rm.rmat_batch_add_tile(b, lv, 1, 0, 10, 5, 0, 0, 8)    # per-level table
    rm.rmat_batch_add_tile(b, t, 1, 0, 10, 4, 15, 3, 8)
    assert rm.rmat_batch_size(b) == (1, 10)


THETA3 = np.array([[0.40, 0.15, 0.05], [0.12, 0.10, 0.04], [0.06, 0.03, 0.05]])
THETA3 = THETA3 / THETA3.sum()


def _theta(n0, seed):
    th = np.random.default_rng(seed).dirichlet(np.linspace(4.0, 0.5, n0 * n0)).reshape(n0, n0)
    return th / th.sum()


def _kron_digits(key, n0, L):
    """Symbols of a library Kronecker path key (base-n0^2 digits, left-aligned
    in D digits, D = the largest with n0^D <= 2^32)."""
    S, D = n0 * n0, 0
    while n0 ** (D + 1) <= 2 ** 32:
        D += 1
    return [int(key) // S ** (D - 1 - t) % S for t in range(L)]


@pytest.mark.parametrize("n0,k,kind,x", [(3, 12, "variable", 500), (3, 40, "variable", 4096), (4, 10, "fixed", 2),
                                         (5, 13, "variable", 4096), (16, 8, "variable", 5000), (3, 7, "fixed", 3)])
def test_kron_table_matches_oracle(n0, k, kind, x):
    th = THETA3 if n0 == 3 else _theta(n0, n0)
    if kind == "variable":
        t, ot = rm.rmat_build_table_kron(th, n0, k, x), oracle.KronTable.variable(th, n0, k, x)
    else:
        t, ot = rm.rmat_build_table_kron_fixed(th, n0, k, x), oracle.KronTable.fixed(th, n0, x)
    ex = rm.rmat_table_export(t)
    assert ex["entries"] == ot.entries and ex["bits"] == ot.bits and ex["max_len"] == ot.max_len
    for f in ("len", "p", "w", "thr", "alias"):
        assert np.array_equal(ex[f], getattr(ot, f)), f
    for i in range(ot.entries):
        L = int(ot.len[i])
        assert _kron_digits(ex["sym"][i], n0, L) == [int(v) for v in ot.sym[i, :L]]
    info = rm.rmat_table_info(t)
    assert info["n0"] == n0
    assert info["index_bytes"] == (4 if n0 ** k <= 2 ** 32 else 8)
    N = 1 << ot.bits
    # packed arrays for the contract-case kernel (A32, P32, 16 powers, 16 magic
    # divisors) when the
    # IDs fit 32 bits and the longest path's digits fit S bits, 2S + 4 <= 32
    S = max(1, (n0 ** int(ot.max_len) - 1).bit_length())
    packs = n0 ** k <= 2 ** 32 and ot.max_len <= 15 and 2 * S + 4 <= 32
    assert info["device_image_bytes"] == 4 * (256 + 2 * N + 4 * N + (2 * N + 32 if packs else 0))


def test_kron_two_by_two_is_the_rmat_table():
    th = np.array([[0.57, 0.19], [0.19, 0.05]])
    a, b = rm.rmat_build_table_kron(th, 2, 26, 4096), rm.rmat_build_table(0.57, 0.19, 0.19, 0.05, 26, 4096)
    ea, eb = rm.rmat_table_export(a), rm.rmat_table_export(b)
    assert all(np.array_equal(ea[f], eb[f]) for f in ("sym", "len", "p", "w", "thr", "alias"))
    assert rm.rmat_table_info(a)["n0"] == 2


def test_kron_host_checks():
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_kron(np.ones(1), 1, 5, 100)
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_kron(np.ones(289) / 289, 17, 5, 1000)
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_kron(THETA3, 3, 41, 100)          # 3^41 > 2^64
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_kron(THETA3, 3, 10, 9)            # bound < n0^2 + 1
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_kron(THETA3 * 1.1, 3, 10, 100)    # does not sum to 1
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_kron_fixed(THETA3, 3, 10, 9)      # 9^9 > 2^24 entries
    t = rm.rmat_build_table_kron(THETA3, 3, 10, 100)
    with pytest.raises(rm.RmatError):
        rm.rmat_table_set_flags(t, rm.RMAT_UNDIRECTED)
    with pytest.raises(rm.RmatError):
        rm.rmat_table_set_scramble(t, True, 1)
    b = rm.rmat_batch_create()
    with pytest.raises(rm.RmatError):
        rm.rmat_batch_add(b, t, 1, 0, 10, 8)
    with pytest.raises(rm.RmatError):
        rm.rmat_partition_create(t, 2, 100, 1)


def test_gpu_table_build_fails_cleanly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_gpu(0.57, 0.19, 0.19, 0.05, 26, 4096)
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_gpu(0.57, 0.19, 0.19, 0.05, 26, 4)   # bound below 5


def test_dedup_host_checks():
    with pytest.raises(rm.RmatError):
        rm.rmat_dedup_edges(8, 10, 32)        # k above 31
    assert rm.rmat_dedup_edges(8, 0, 20) == 0  # nothing to do, no device needed
    rm.rmat_dedup_release()                    # holds nothing: a no-op


def test_selftest_argument_check():
    with pytest.raises(rm.RmatError):
        rm.rmat_selftest_bounded_wait(0)


def test_batch_header_size_matches_the_library():
    """The autotuner's shared-memory budget for batched tables subtracts the
    same header as the batched kernel lays out."""
    from paper_1905_03525_gb300 import autotune
    src = open(os.path.join(ROOT, "paper_1905_03525_gb300", "csrc", "rmat_kernels.h")).read()
    m = re.search(r"constexpr size_t kBatchHeaderBytes = (\d+);", src)
    assert m and int(m.group(1)) == autotune.BATCH_HEADER_BYTES


def _prototypes():
    """(name, [parameter declarations]) of every function in include/*.h."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", fn)).read(), flags=re.S)
        for m in re.finditer(r"(rmat_[A-Za-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
            params = [p.strip() for p in m.group(2).split(",")]
            out[m.group(1)] = [] if params == ["void"] or params == [""] else params
    return out


def test_binding_signatures_match_the_header():
    """Every prototype's parameters have the ctypes types the binding declares
    (pointer and handle -> void*, double, int, unsigned / uint32_t, uint64_t)."""
    c = ctypes

    def kind(decl):
        if "*" in decl or decl.startswith("rmat_stream_t"):
            return c.c_void_p
        t = decl.replace("const ", "").split()[0]
        return {"double": c.c_double, "int": c.c_int, "unsigned": c.c_uint, "uint32_t": c.c_uint,
                "uint64_t": c.c_uint64}.get(t)

    protos = _prototypes()
    sigs = {name: args for name, _, args in _capi.SIGNATURES}
    checked = 0
    for name, params in protos.items():
        if name not in sigs:
            continue
        assert len(params) == len(sigs[name]), (name, params)
        for decl, bound in zip(params, sigs[name]):
            want = kind(decl)
            if want is not None:
                assert ctypes.sizeof(want) == ctypes.sizeof(bound) and (want is c.c_double) == (bound is c.c_double), \
                    (name, decl, bound)
        checked += 1
    assert checked == len(protos) == len(declared_functions())
