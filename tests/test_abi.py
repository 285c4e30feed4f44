"""The C-ABI library loads, exports every symbol include/qmc.h declares, and
rejects invalid arguments on the host before touching CUDA.  CPU only: no
call here reaches a kernel launch."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import build

    build.build()
    from paper_2307_15584_gb300 import binding

    return binding


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "qmc.h")).read()
    return sorted(set(re.findall(r"QMC_API\s+[\w\s\*]+?\b(qmc_\w+)\s*\(", text)))


def test_header_symbols_exported(B):
    declared = _declared_symbols()
    assert len(declared) >= 11
    lib = ctypes.CDLL(B.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTED) == sorted(declared)
    checked = ctypes.CDLL(os.path.join(os.path.dirname(B.LIB_PATH), "libqmc_gb300_checked.so"))
    for name in declared:  # the checked build exports the same interface
        assert hasattr(checked, name), name
    assert B.qmc_abi_version() == 5
    assert ctypes.sizeof(B.qmc_problem) == 72  # 4 + 3 pointers + 8 words, as in include/qmc.h
    assert "INVALID" in B.qmc_status_string(1)


def test_sobol_matrices_match_oracle(B, oracle):
    """The library's host construction (Bratley-Fox form, primitivity by the
    order test with prime factors) equals the oracle's (m-integer form, brute
    order search) for every dimension it supports."""
    raw = inputs.sobol_raw_init(37, seed=123)
    got = B.qmc_sobol_matrices(37, raw)
    np.testing.assert_array_equal(got, oracle.sobol_matrices(37, raw))
    with pytest.raises(B.QMCError):
        B.qmc_sobol_matrices(38, inputs.sobol_raw_init(38))
    with pytest.raises(B.QMCError):
        B.qmc_sobol_matrices(0, raw)


def test_wide_sobol_matrices_match_oracle(B, oracle):
    """Wide columns (Alg. 3): the library's truncated-word recurrence equals the
    oracle's exact 128-bit direction numbers for every m in 32..64."""
    raw = inputs.sobol_raw_init(37, seed=321)
    for m in (32, 33, 52, 63, 64):
        np.testing.assert_array_equal(B.qmc_sobol_matrices_wide(37, m, raw), oracle.sobol_matrices_wide(37, m, raw))
    np.testing.assert_array_equal(B.qmc_sobol_matrices_wide(37, 32, raw), B.qmc_sobol_matrices(37, raw))
    for m in (31, 65):
        with pytest.raises(B.QMCError):
            B.qmc_sobol_matrices_wide(4, m, raw)


FAKE = 0x10000  # an aligned non-null "device" address: never dereferenced (calls fail validation)


def _status(fn, *args):
    return fn(*args)


def test_points_validation(B):
    L = B._lib
    S = None
    # null matrices / no outputs / bad scramble / missing seeds
    assert L.qmc_sobol_points(None, 4, 0, 16, 0, None, FAKE, None, S) == 1
    assert L.qmc_sobol_points(FAKE, 4, 0, 16, 0, None, None, None, S) == 1
    assert L.qmc_sobol_points(FAKE, 4, 0, 16, 4, FAKE, FAKE, None, S) == 1
    assert L.qmc_sobol_points(FAKE, 4, 0, 16, 2, None, FAKE, None, S) == 1
    assert L.qmc_sobol_points(FAKE, 0, 0, 16, 0, None, FAKE, None, S) == 1
    assert L.qmc_sobol_points(FAKE, 1025, 0, 16, 0, None, FAKE, None, S) == 1
    # index range beyond 2^32 (Sec. 2.5: no silent wrap-around)
    assert L.qmc_sobol_points(FAKE, 4, (1 << 32) - 8, 9, 0, None, FAKE, None, S) == 2
    assert L.qmc_sobol_points(FAKE, 4, 1 << 33, 1, 0, None, FAKE, None, S) == 2
    # misaligned outputs
    assert L.qmc_sobol_points(FAKE, 4, 0, 16, 0, None, FAKE + 2, None, S) == 3
    assert L.qmc_lattice_points(FAKE, None, 4, 0, 16, 0, None, FAKE + 1, S) == 3
    # lattice flags / generator
    assert L.qmc_lattice_points(None, None, 4, 0, 16, 0, FAKE, None, S) == 1
    assert L.qmc_lattice_points(FAKE, None, 4, 0, 16, 2, FAKE, None, S) == 1
    # count = 0 is a no-op that needs no device
    assert L.qmc_sobol_points(FAKE, 4, 0, 0, 0, None, FAKE, None, S) == 0
    assert L.qmc_lattice_points(FAKE, None, 4, 1 << 32, 0, 0, FAKE, None, S) == 0


def test_wide_and_partitioned_validation(B):
    L = B._lib
    S = None
    U64 = (1 << 64) - 1
    W, Pt, H = L.qmc_sobol_points_wide, L.qmc_sobol_points_partitioned, L.qmc_halton_points_partitioned
    # columns per dimension, dimensions, scramble
    for m in (31, 65):
        assert W(FAKE, m, 4, 0, 16, 0, None, FAKE, None, S) == 1
    assert W(FAKE, 64, 0, 0, 16, 0, None, FAKE, None, S) == 1
    assert W(FAKE, 64, 4, 0, 16, 2, None, FAKE, None, S) == 1
    # ranges end at 2^m (m = 64: at 2^64 - 1, with no wrap of begin + count)
    assert W(FAKE, 40, 4, (1 << 40) - 8, 9, 0, None, FAKE, None, S) == 2
    assert W(FAKE, 64, 4, U64 - 3, 5, 0, None, FAKE, None, S) == 2
    assert W(FAKE, 64, 4, U64, 2, 0, None, FAKE, None, S) == 2
    assert W(FAKE, 64, 1 << 10, 0, 1 << 53, 0, None, FAKE, None, S) == 2  # output offsets beyond 2^62
    assert W(FAKE, 40, 4, 1 << 40, 0, 0, None, FAKE, None, S) == 0
    # partition: q < m, p < 2^q, J below 2^(m-q)
    assert Pt(FAKE, 40, 4, 40, 0, 0, 16, 0, None, FAKE, None, S) == 1
    assert Pt(FAKE, 40, 4, 3, 8, 0, 16, 0, None, FAKE, None, S) == 1
    assert Pt(FAKE, 40, 4, 3, 7, (1 << 37) - 4, 5, 0, None, FAKE, None, S) == 2
    assert Pt(FAKE, 64, 4, 63, 1, 2, 1, 0, None, FAKE, None, S) == 2
    assert Pt(FAKE, 64, 4, 3, 7, 0, 0, 0, None, FAKE, None, S) == 0
    assert Pt(FAKE, 64, 4, 3, 7, 0, 16, 0, None, FAKE + 2, None, S) == 3
    # Halton partition: s <= 63 output dimensions, q <= 63, p < 2^q
    assert H(64, 0, None, 2, 0, 0, 16, FAKE, None, S) == 1
    assert H(0, 0, None, 2, 0, 0, 16, FAKE, None, S) == 1
    assert H(4, 0, None, 64, 0, 0, 16, FAKE, None, S) == 1
    assert H(4, 0, None, 2, 4, 0, 16, FAKE, None, S) == 1
    assert H(4, 2, None, 2, 0, 0, 16, FAKE, None, S) == 1
    m3 = np.array([3, 1, 1, 1], np.uint32)  # 3 is not a unit modulo the base 3
    assert H(4, 2, m3.ctypes.data, 2, 0, 0, 16, FAKE, None, S) == 1
    assert H(4, 0, None, 2, 0, 1 << 62, 1, FAKE, None, S) == 2


def _problem(B, **kw):
    d = dict(source=B.SOURCE_SOBOL, integrand=B.F_GAUSSMIX4_6D, s=6, randomize=B.SCRAMBLE_NESTED,
             matrices=FAKE, seeds=FAKE, seeds_per_integral=True, max_count=65536)
    d.update(kw)
    return B.make_problem(**d)


def test_workspace_sizing(B):
    p = _problem(B)
    counts = inputs.log_uniform_counts(1000)
    exact = B.qmc_integrate_workspace_bytes(p, 1000, counts)
    worst = B.qmc_integrate_workspace_bytes(p, 1000, None)
    assert 0 < exact < worst
    pg = _problem(B, with_gradient=True)
    assert B.qmc_integrate_workspace_bytes(pg, 1000, counts) > exact
    assert B.qmc_integrate_workspace_bytes(_problem(B, s=5), 10, None) == 0  # mixture needs s = 6
    assert B.qmc_integrate_workspace_bytes(_problem(B, chunk=100), 10, None) == 0  # not a power of two


def test_integrate_validation(B):
    L = B._lib
    ref = ctypes.byref
    ws = 1 << 20  # fake 256-aligned address
    p = _problem(B)
    assert L.qmc_integrate(None, 4, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 1
    assert L.qmc_integrate(ref(p), 4, None, FAKE, FAKE, ws, 1 << 30, None) == 1
    assert L.qmc_integrate(ref(p), 4, FAKE, None, FAKE, ws, 1 << 30, None) == 1  # mixture needs theta
    assert L.qmc_integrate(ref(p), 4, FAKE, FAKE + 4, FAKE, ws, 1 << 30, None) == 3
    assert L.qmc_integrate(ref(p), 4, FAKE, FAKE, FAKE, ws + 16, 1 << 30, None) == 7
    assert L.qmc_integrate(ref(p), 4, FAKE, FAKE, FAKE, ws, 64, None) == 7
    for bad in (dict(s=7), dict(integrand=9), dict(source=3), dict(randomize=5), dict(matrices=None),
                dict(seeds=None), dict(block=48), dict(block=512), dict(chunk=16), dict(chunk=16384),
                dict(integrand=B.F_BILINEAR2D, s=6), dict(integrand=B.F_GENZ_OSCILLATORY, s=17)):
        assert L.qmc_integrate(ref(_problem(B, **bad)), 4, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 1, bad
    # backward / fused need the mixture and their outputs
    pg = _problem(B, integrand=B.F_GENZ_PRODUCT_PEAK, s=16)
    assert L.qmc_integrate_backward(ref(pg), 4, FAKE, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 6
    assert L.qmc_integrate_backward(ref(p), 4, FAKE, FAKE, None, FAKE, ws, 1 << 30, None) == 1
    assert L.qmc_integrate_fwd_bwd(ref(p), 4, FAKE, FAKE, FAKE, FAKE, FAKE, None, ws, 1 << 30, None) == 1
    assert L.qmc_integrate_points(ref(p), 4, FAKE, None, 0, FAKE, FAKE, ws, 1 << 30, None) == 1
    assert L.qmc_integrate_points(ref(p), 4, FAKE, FAKE, 2, FAKE, FAKE, ws, 1 << 30, None) == 1
    # n = 0 with valid arguments is a no-op
    assert L.qmc_integrate(ref(p), 0, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 0
    assert L.qmc_read_device_error(None, ctypes.byref(ctypes.c_uint32()), None) == 1


def test_runtime_validation(B):
    L = B._lib
    assert L.qmc_graph_begin(None) == 1  # the legacy default stream cannot be captured
    assert L.qmc_graph_end(None, None) == 1
    assert L.qmc_graph_launch(None, None) == 1
    assert L.qmc_graph_destroy(None) == 1
    assert L.qmc_tune_clear() == 0
    best = B.qmc_tuning()
    assert L.qmc_tune_integrate(None, 4, FAKE, FAKE, None, FAKE, None, None, FAKE, 1 << 20, None,
                                ctypes.byref(best)) == 1
    p = _problem(B)
    # forward+backward tuning needs a target and a loss buffer
    assert L.qmc_tune_integrate(ctypes.byref(p), 4, FAKE, FAKE, None, FAKE, FAKE, None, FAKE, 1 << 20, None,
                                ctypes.byref(best)) == 1


def test_random_lattice_validation(B):
    L = B._lib
    S = None
    R = L.qmc_random_lattice_points
    for bad in ((2, 7, 4, 8, 64, 64, 0, 16, 4), (0, 7, 3, 8, 64, 64, 0, 16, 4), (0, 7, 32, 8, 64, 64, 0, 16, 4),
                (0, 7, 0, 8, 64, 64, 0, 16, 4), (0, 7, 4, 0, 64, 64, 0, 16, 4), (0, 7, 4, 1025, 64, 64, 0, 16, 4),
                (0, 7, 4, 8, (1 << 20) + 1, 1, 0, 16, 4), (0, 7, 4, 8, 64, 64, 0, 16, 0)):
        assert R(*bad, FAKE, None, S) == 1, bad
    assert R(0, 7, 4, 8, 64, 64, 4090, 7, 4, FAKE, None, S) == 2  # beyond the image
    assert R(0, 7, 4, 8, 64, 64, 4096, 0, 4, FAKE, None, S) == 0  # empty range: no launch
    assert R(0, 7, 4, 8, 64, 64, 0, 16, 4, FAKE + 2, None, S) == 3
    ref = ctypes.byref
    ws = 1 << 20
    base = dict(source=B.SOURCE_RANDOM_LATTICE, randomize=B.rlat_randomize(B.RLAT_HASH, 4), image_width=64,
                seeds_per_integral=False)
    for bad in (dict(randomize=B.rlat_randomize(2, 4)), dict(randomize=B.rlat_randomize(0, 3)),
                dict(randomize=B.rlat_randomize(0, 32)), dict(seeds=None), dict(image_width=0),
                dict(image_width=(1 << 20) + 1)):
        kw = dict(base)
        kw.update(bad)
        assert L.qmc_integrate(ref(_problem(B, **kw)), 4, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 1, bad


def test_partitioned_integration_validation(B):
    """Sec. 2.5.1 integration: 32..64 columns, q <= 32 with m >= 32 + q, Sobol' only."""
    L = B._lib
    ref = ctypes.byref
    ws = 1 << 20
    for bad in (dict(index_bits=31), dict(index_bits=65), dict(index_bits=0, partition_log2=1),
                dict(index_bits=40, partition_log2=9), dict(index_bits=64, partition_log2=33),
                dict(source=B.SOURCE_LATTICE, g=FAKE, randomize=0, index_bits=64),
                dict(source=B.SOURCE_LATTICE, g=FAKE, randomize=0, partition_log2=1)):
        assert L.qmc_integrate(ref(_problem(B, **bad)), 4, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 1, bad
        assert B.qmc_integrate_workspace_bytes(_problem(B, **bad), 4, None) == 0, bad
    for good in (dict(index_bits=32), dict(index_bits=40, partition_log2=8), dict(index_bits=64, partition_log2=32)):
        assert B.qmc_integrate_workspace_bytes(_problem(B, **good), 4, None) > 0, good
        assert L.qmc_integrate(ref(_problem(B, **good)), 0, FAKE, FAKE, FAKE, ws, 1 << 30, None) == 0, good


def test_fault_injection_on_host(B, monkeypatch):
    """QMC_FAULT_INJECT=launch: every entry point that would enqueue GPU work
    validates its arguments, then fails its launch on the host with QMC_ERR_CUDA
    and records QMC_INJECTED_FAULT as the thread's last CUDA error -- without a
    GPU (this runs on the CPU) and therefore without any fault on one."""
    L = B._lib
    ref = ctypes.byref
    ws = 1 << 20
    monkeypatch.setenv("QMC_FAULT_INJECT", "launch")
    p = _problem(B)
    static = _problem(B, max_count=4096)
    best = B.qmc_tuning()
    calls = {
        "qmc_sobol_points": lambda: L.qmc_sobol_points(FAKE, 4, 0, 16, 3, FAKE, FAKE, None, 0),
        "qmc_sobol_points_wide": lambda: L.qmc_sobol_points_wide(FAKE, 64, 4, 1 << 40, 16, 2, FAKE, FAKE, None, 0),
        "qmc_sobol_points_partitioned": lambda: L.qmc_sobol_points_partitioned(FAKE, 64, 4, 3, 5, 0, 16, 0, None,
                                                                               FAKE, None, 0),
        "qmc_lattice_points": lambda: L.qmc_lattice_points(FAKE, None, 4, 0, 16, 0, FAKE, None, 0),
        "qmc_halton_points": lambda: L.qmc_halton_points(4, 1, None, 0, 16, FAKE, None, 0),
        "qmc_halton_points_partitioned": lambda: L.qmc_halton_points_partitioned(4, 0, None, 2, 1, 0, 16, FAKE,
                                                                                 None, 0),
        "qmc_pixel_lattice_points": lambda: L.qmc_pixel_lattice_points(FAKE, 4, 8, 8, 0, 4, 2, FAKE, None, 0),
        "qmc_random_lattice_points": lambda: L.qmc_random_lattice_points(0, 7, 4, 8, 64, 64, 0, 16, 4, FAKE,
                                                                         None, 0),
        "qmc_integrate": lambda: L.qmc_integrate(ref(p), 4, FAKE, FAKE, FAKE, ws, 1 << 30, 0),
        "qmc_integrate_backward": lambda: L.qmc_integrate_backward(ref(p), 4, FAKE, FAKE, FAKE, FAKE, ws,
                                                                   1 << 30, 0),
        "qmc_integrate_fwd_bwd": lambda: L.qmc_integrate_fwd_bwd(ref(p), 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, ws,
                                                                 1 << 30, 0),
        "qmc_integrate_points": lambda: L.qmc_integrate_points(ref(p), 4, FAKE, FAKE, 0, FAKE, FAKE, ws, 1 << 30, 0),
        "qmc_integrate_static": lambda: L.qmc_integrate_static(ref(static), 4, FAKE, FAKE, FAKE, 0),
        "qmc_read_device_error": lambda: L.qmc_read_device_error(ws, ref(ctypes.c_uint32()), 0),
        "qmc_tune_integrate": lambda: L.qmc_tune_integrate(ref(p), 4, FAKE, FAKE, None, FAKE, None, None, ws,
                                                           1 << 30, 0, ref(best)),
    }
    for name, call in calls.items():
        assert call() == 4, name
        assert B.qmc_last_cuda_error() == B.QMC_INJECTED_FAULT, name
    # argument errors still come first
    assert L.qmc_sobol_points(None, 4, 0, 16, 0, None, FAKE, None, 0) == 1
    assert L.qmc_integrate(ref(p), 4, FAKE, FAKE, FAKE, ws + 16, 1 << 30, 0) == 7
    # any other value of the variable injects nothing: validation-only paths still succeed
    monkeypatch.setenv("QMC_FAULT_INJECT", "none")
    assert L.qmc_sobol_points(FAKE, 4, 0, 0, 0, None, FAKE, None, 0) == 0


def test_autotune_cache_file(B, tmp_path):
    """The tuner's records round-trip through the JSON cache file: valid entries
    load, malformed ones are skipped, a saved file loads back to the same records,
    and a lookup finds the record of the current device kind (on a machine without
    a GPU that kind is the empty name with 0 SMs)."""
    src = tmp_path / "in.json"
    entry = ('{{"device": "{dev}", "sms": {sms}, "source": 0, "integrand": 3, "s": 6, "randomize": 2, '
             '"seeds_per_integral": 1, "gradient": {g}, "size_class": 10, "chunk": {c}, "block": {b}}}')
    src.write_text('{"qmc_autotune_cache": 1, "entries": [\n' + ",\n".join([
        entry.format(dev="", sms=0, g=0, c=2048, b=128),
        entry.format(dev="NVIDIA GB300", sms=152, g=1, c=4096, b=256),
        entry.format(dev="", sms=0, g=1, c=100, b=256),  # not a power of two: skipped
        '{"device": "", "sms": 0, "chunk": 1024}',  # incomplete: skipped
    ]) + "\n]}\n")
    B.qmc_tune_clear()
    assert B.qmc_tune_load(str(src)) == 2
    p = _problem(B)
    hit = B.qmc_tune_lookup(p, 1000)  # size class ceil(log2 1000) = 10
    assert (hit.chunk, hit.block) == (2048, 128)
    assert B.qmc_tune_lookup(p, 1000, with_gradient=True).chunk == 0  # recorded for another device kind
    assert B.qmc_tune_lookup(p, 5000).chunk == 0  # another size class
    out = tmp_path / "out.json"
    B.qmc_tune_save(str(out))
    import json
    saved = json.loads(out.read_text())["entries"]
    assert sorted((e["device"], e["gradient"], e["chunk"], e["block"]) for e in saved) == \
        [("", 0, 2048, 128), ("NVIDIA GB300", 1, 4096, 256)]
    B.qmc_tune_clear()
    assert B.qmc_tune_lookup(p, 1000).chunk == 0
    assert B.qmc_tune_load(str(out)) == 2
    assert B.qmc_tune_lookup(p, 1000).chunk == 2048
    B.qmc_tune_clear()
    with pytest.raises(B.QMCError) as e:
        B.qmc_tune_load(str(tmp_path / "missing.json"))
    assert e.value.status == 8
    with pytest.raises(B.QMCError) as e:
        B.qmc_tune_save(str(tmp_path / "no_such_dir" / "x.json"))
    assert e.value.status == 8


def test_checked_error_word_only_in_the_checked_build(B):
    """The normal build has no error word: qmc_checked_error answers QMC_ERR_UNSUPPORTED
    (with no CUDA call, so this runs on the CPU) and reports 0 bits."""
    bits = ctypes.c_uint32(123)
    assert B._lib.qmc_checked_error(ctypes.byref(bits), 0) == 6
    assert bits.value == 0
    assert B._lib.qmc_checked_error(None, 0) == 1
