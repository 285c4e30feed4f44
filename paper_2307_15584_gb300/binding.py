"""ctypes binding of libqmc_gb300.so (include/qmc.h): argument marshalling only.

Every function named ``qmc_*`` here calls the C entry point of the same name
with device pointers taken from torch tensors and the current torch CUDA
stream.  Nothing is computed in Python and there is no CPU fallback: importing
this module raises when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_double, c_size_t, c_uint32, c_uint64, c_void_p

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
CHECKED = os.environ.get("QMC_CHECKED") == "1"  # the checked build: bounds-tested stores (include/qmc.h)
LIB_PATH = os.path.join(_PKG, "libqmc_gb300_checked.so" if CHECKED else "libqmc_gb300.so")
if not os.path.exists(LIB_PATH):
    raise RuntimeError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`; "
        "the QMC path has no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

# enums of include/qmc.h
QMC_OK = 0
STATUS_NAMES = {0: "QMC_OK", 1: "QMC_ERR_INVALID_ARG", 2: "QMC_ERR_RANGE", 3: "QMC_ERR_ALIGN",
                4: "QMC_ERR_CUDA", 5: "QMC_ERR_TIMEOUT", 6: "QMC_ERR_UNSUPPORTED", 7: "QMC_ERR_WORKSPACE",
                8: "QMC_ERR_IO"}
QMC_INJECTED_FAULT = -1
SCRAMBLE_NONE, SCRAMBLE_XOR, SCRAMBLE_NESTED, SCRAMBLE_NESTED_XOR = 0, 1, 2, 3
LATTICE_BACKWARD = 1
SOURCE_SOBOL, SOURCE_LATTICE, SOURCE_PIXEL_LATTICE, SOURCE_RANDOM_LATTICE = 0, 1, 2, 3
RLAT_HASH, RLAT_LFSR = 0, 1
F_BILINEAR2D, F_GENZ_PRODUCT_PEAK, F_GENZ_OSCILLATORY, F_GAUSSMIX4_6D, F_SCENE4D = 0, 1, 2, 3, 4

EXPORTED = ["qmc_abi_version", "qmc_status_string", "qmc_sobol_matrices", "qmc_sobol_points",
            "qmc_lattice_points", "qmc_integrate_workspace_bytes", "qmc_integrate",
            "qmc_integrate_backward", "qmc_integrate_fwd_bwd", "qmc_integrate_points",
            "qmc_read_device_error", "qmc_integrate_static", "qmc_tune_integrate", "qmc_tune_clear",
            "qmc_graph_begin", "qmc_graph_end", "qmc_graph_launch", "qmc_graph_destroy",
            "qmc_pixel_lattice_points", "qmc_halton_points", "qmc_sobol_matrices_wide",
            "qmc_sobol_points_wide", "qmc_sobol_points_partitioned", "qmc_halton_points_partitioned",
            "qmc_random_lattice_points", "qmc_last_cuda_error", "qmc_tune_save", "qmc_tune_load",
            "qmc_tune_lookup", "qmc_checked_error"]
HALTON_PLAIN, HALTON_FAURE, HALTON_LINEAR = 0, 1, 2


class QMCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.qmc_status_string(status).decode()
        super().__init__(f"{where}: {msg}")


class qmc_tuning(ctypes.Structure):
    _fields_ = [("chunk", c_uint32), ("block", c_uint32), ("ms", ctypes.c_float)]


class qmc_problem(ctypes.Structure):
    _fields_ = [("source", c_uint32), ("integrand", c_uint32), ("s", c_uint32), ("randomize", c_uint32),
                ("d_matrices", c_void_p), ("d_g", c_void_p), ("d_seeds", c_void_p),
                ("seeds_per_integral", c_uint32), ("chunk", c_uint32), ("block", c_uint32),
                ("max_count", c_uint32), ("with_gradient", c_uint32), ("image_width", c_uint32),
                ("index_bits", c_uint32), ("partition_log2", c_uint32)]


_P = c_void_p
_sigs = {
    "qmc_abi_version": (c_uint32, []),
    "qmc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qmc_sobol_matrices": (ctypes.c_int, [c_uint32, _P, _P]),
    "qmc_sobol_points": (ctypes.c_int, [_P, c_uint32, c_uint64, c_uint64, c_uint32, _P, _P, _P, _P]),
    "qmc_lattice_points": (ctypes.c_int, [_P, _P, c_uint32, c_uint64, c_uint64, c_uint32, _P, _P, _P]),
    "qmc_pixel_lattice_points": (ctypes.c_int, [_P, c_uint32, c_uint32, c_uint32, c_uint64, c_uint64, c_uint32,
                                                _P, _P, _P]),
    "qmc_halton_points": (ctypes.c_int, [c_uint32, c_uint32, _P, c_uint64, c_uint64, _P, _P, _P]),
    "qmc_sobol_matrices_wide": (ctypes.c_int, [c_uint32, c_uint32, _P, _P]),
    "qmc_random_lattice_points": (ctypes.c_int, [c_uint32, c_uint32, c_uint32, c_uint32, c_uint32, c_uint32,
                                                 c_uint64, c_uint64, c_uint32, _P, _P, _P]),
    "qmc_sobol_points_wide": (ctypes.c_int, [_P, c_uint32, c_uint32, c_uint64, c_uint64, c_uint32, _P, _P, _P,
                                             _P]),
    "qmc_sobol_points_partitioned": (ctypes.c_int, [_P, c_uint32, c_uint32, c_uint32, c_uint64, c_uint64,
                                                    c_uint64, c_uint32, _P, _P, _P, _P]),
    "qmc_halton_points_partitioned": (ctypes.c_int, [c_uint32, c_uint32, _P, c_uint32, c_uint64, c_uint64,
                                                     c_uint64, _P, _P, _P]),
    "qmc_integrate_workspace_bytes": (c_size_t, [ctypes.POINTER(qmc_problem), c_uint32, _P]),
    "qmc_integrate": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, _P, _P, _P, _P, c_size_t, _P]),
    "qmc_integrate_backward": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, _P, _P, _P, _P, _P,
                                              c_size_t, _P]),
    "qmc_integrate_fwd_bwd": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, _P, _P, _P, _P, _P, _P,
                                             _P, c_size_t, _P]),
    "qmc_integrate_points": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, _P, _P, c_uint32, _P, _P,
                                            _P, c_size_t, _P]),
    "qmc_read_device_error": (ctypes.c_int, [_P, ctypes.POINTER(c_uint32), _P]),
    "qmc_integrate_static": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, _P, _P, _P, _P]),
    "qmc_tune_integrate": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, _P, _P, _P, _P, _P, _P, _P,
                                          c_size_t, _P, ctypes.POINTER(qmc_tuning)]),
    "qmc_tune_clear": (ctypes.c_int, []),
    "qmc_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "qmc_tune_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(c_uint32)]),
    "qmc_tune_lookup": (ctypes.c_int, [ctypes.POINTER(qmc_problem), c_uint32, c_uint32,
                                       ctypes.POINTER(qmc_tuning)]),
    "qmc_last_cuda_error": (ctypes.c_int, []),
    "qmc_checked_error": (ctypes.c_int, [ctypes.POINTER(c_uint32), c_uint32]),
    "qmc_graph_begin": (ctypes.c_int, [_P]),
    "qmc_graph_end": (ctypes.c_int, [_P, ctypes.POINTER(c_void_p)]),
    "qmc_graph_launch": (ctypes.c_int, [c_void_p, _P]),
    "qmc_graph_destroy": (ctypes.c_int, [c_void_p]),
}
for _name, (_res, _args) in _sigs.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _check(status: int, where: str) -> None:
    if status != QMC_OK:
        raise QMCError(status, where)


def _dev(t):
    """Device pointer of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def u32_tensor(a, device="cuda") -> torch.Tensor:
    """uint32 numpy data as an int32 tensor holding the same bits."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


def as_u32(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


# ----------------------------------------------------------------- C entry points
def qmc_abi_version() -> int:
    return _lib.qmc_abi_version()


def qmc_status_string(status: int) -> str:
    return _lib.qmc_status_string(status).decode()


def qmc_last_cuda_error() -> int:
    """cudaError_t code behind this thread's most recent QMC_ERR_CUDA (QMC_INJECTED_FAULT
    for a fault injected with QMC_FAULT_INJECT=launch)."""
    return _lib.qmc_last_cuda_error()


def qmc_sobol_matrices(s: int, raw_init) -> np.ndarray:
    raw = np.ascontiguousarray(raw_init, dtype=np.uint32)
    out = np.zeros((s, 32), np.uint32)
    _check(_lib.qmc_sobol_matrices(s, raw.ctypes.data if raw.size else None, out.ctypes.data),
           "qmc_sobol_matrices")
    return out


def qmc_sobol_matrices_wide(s: int, m: int, raw_init) -> np.ndarray:
    raw = np.ascontiguousarray(raw_init, dtype=np.uint32)
    out = np.zeros((s, m), np.uint32)
    _check(_lib.qmc_sobol_matrices_wide(s, m, raw.ctypes.data if raw.size else None, out.ctypes.data),
           "qmc_sobol_matrices_wide")
    return out


def qmc_sobol_points_wide(matrices, m, s, index_begin, count, scramble, seeds, out_u32, out_f32, stream=None):
    _check(_lib.qmc_sobol_points_wide(_dev(matrices), m, s, index_begin, count, scramble, _dev(seeds),
                                      _dev(out_u32), _dev(out_f32), _stream(stream)), "qmc_sobol_points_wide")


def qmc_sobol_points_partitioned(matrices, m, s, q, p, j_begin, count, scramble, seeds, out_u32, out_f32,
                                 stream=None):
    _check(_lib.qmc_sobol_points_partitioned(_dev(matrices), m, s, q, p, j_begin, count, scramble, _dev(seeds),
                                             _dev(out_u32), _dev(out_f32), _stream(stream)),
           "qmc_sobol_points_partitioned")


def qmc_sobol_points(matrices, s, index_begin, count, scramble, seeds, out_u32, out_f32, stream=None):
    _check(_lib.qmc_sobol_points(_dev(matrices), s, index_begin, count, scramble, _dev(seeds), _dev(out_u32),
                                 _dev(out_f32), _stream(stream)), "qmc_sobol_points")


def qmc_pixel_lattice_points(g, s, image_width, image_height, pixel_begin, n_pixels, spp, out_u32, out_f32,
                             stream=None):
    _check(_lib.qmc_pixel_lattice_points(_dev(g), s, image_width, image_height, pixel_begin, n_pixels, spp,
                                         _dev(out_u32), _dev(out_f32), _stream(stream)), "qmc_pixel_lattice_points")


def qmc_halton_points(s, mode, multipliers, index_begin, count, out_u32, out_f32, stream=None):
    """multipliers: host array [s] for HALTON_LINEAR, else None."""
    m = None if multipliers is None else np.ascontiguousarray(multipliers, dtype=np.uint32)
    _check(_lib.qmc_halton_points(s, mode, None if m is None else m.ctypes.data, index_begin, count,
                                  _dev(out_u32), _dev(out_f32), _stream(stream)), "qmc_halton_points")


def qmc_random_lattice_points(kind, seed, instances, s, image_width, image_height, pixel_begin, n_pixels, spp,
                              out_u32, out_f32, stream=None):
    _check(_lib.qmc_random_lattice_points(kind, seed, instances, s, image_width, image_height, pixel_begin,
                                          n_pixels, spp, _dev(out_u32), _dev(out_f32), _stream(stream)),
           "qmc_random_lattice_points")


def rlat_randomize(kind: int, instances: int) -> int:
    """qmc_problem.randomize of QMC_SOURCE_RANDOM_LATTICE."""
    return kind | (instances << 8)


def qmc_halton_points_partitioned(s, mode, multipliers, q, p, j_begin, count, out_u32, out_f32, stream=None):
    """multipliers: host array [s] (bases 3, 5, ..) for HALTON_LINEAR, else None."""
    m = None if multipliers is None else np.ascontiguousarray(multipliers, dtype=np.uint32)
    _check(_lib.qmc_halton_points_partitioned(s, mode, None if m is None else m.ctypes.data, q, p, j_begin, count,
                                              _dev(out_u32), _dev(out_f32), _stream(stream)),
           "qmc_halton_points_partitioned")


def qmc_lattice_points(g, shift, s, index_begin, count, flags, out_u32, out_f32, stream=None):
    _check(_lib.qmc_lattice_points(_dev(g), _dev(shift), s, index_begin, count, flags, _dev(out_u32),
                                   _dev(out_f32), _stream(stream)), "qmc_lattice_points")


def qmc_integrate_workspace_bytes(problem: qmc_problem, n_integrals: int, h_counts=None) -> int:
    hc = None if h_counts is None else np.ascontiguousarray(h_counts, dtype=np.uint32)
    return _lib.qmc_integrate_workspace_bytes(ctypes.byref(problem), n_integrals,
                                              None if hc is None else hc.ctypes.data)


def qmc_integrate(problem, n_integrals, counts, theta, estimate, workspace, workspace_bytes=None, stream=None):
    wb = workspace.numel() * workspace.element_size() if workspace_bytes is None else workspace_bytes
    _check(_lib.qmc_integrate(ctypes.byref(problem), n_integrals, _dev(counts), _dev(theta), _dev(estimate),
                              _dev(workspace), wb, _stream(stream)), "qmc_integrate")


def qmc_integrate_backward(problem, n_integrals, counts, theta, grad_estimate, grad_theta, workspace,
                           workspace_bytes=None, stream=None):
    wb = workspace.numel() * workspace.element_size() if workspace_bytes is None else workspace_bytes
    _check(_lib.qmc_integrate_backward(ctypes.byref(problem), n_integrals, _dev(counts), _dev(theta),
                                       _dev(grad_estimate), _dev(grad_theta), _dev(workspace), wb,
                                       _stream(stream)), "qmc_integrate_backward")


def qmc_integrate_fwd_bwd(problem, n_integrals, counts, theta, target, estimate, grad_theta, loss, workspace,
                          workspace_bytes=None, stream=None):
    wb = workspace.numel() * workspace.element_size() if workspace_bytes is None else workspace_bytes
    _check(_lib.qmc_integrate_fwd_bwd(ctypes.byref(problem), n_integrals, _dev(counts), _dev(theta),
                                      _dev(target), _dev(estimate), _dev(grad_theta), _dev(loss),
                                      _dev(workspace), wb, _stream(stream)), "qmc_integrate_fwd_bwd")


def qmc_integrate_points(problem, n_integrals, counts, points, points_shared, theta, estimate, workspace,
                         workspace_bytes=None, stream=None):
    wb = workspace.numel() * workspace.element_size() if workspace_bytes is None else workspace_bytes
    _check(_lib.qmc_integrate_points(ctypes.byref(problem), n_integrals, _dev(counts), _dev(points),
                                     int(points_shared), _dev(theta), _dev(estimate), _dev(workspace), wb,
                                     _stream(stream)), "qmc_integrate_points")


def qmc_integrate_static(problem, n_integrals, counts, theta, estimate, stream=None):
    """qmc_integrate without a workspace argument, for callers that cannot allocate
    device memory: the library integrates in its own fixed device array (see
    include/qmc.h for the size limit and the rule that calls on a device must not
    overlap)."""
    _check(_lib.qmc_integrate_static(ctypes.byref(problem), n_integrals, _dev(counts), _dev(theta),
                                     _dev(estimate), _stream(stream)), "qmc_integrate_static")


def qmc_tune_integrate(problem, n_integrals, counts, theta, estimate, workspace, target=None, grad_theta=None,
                       loss=None, workspace_bytes=None, stream=None) -> qmc_tuning:
    wb = workspace.numel() * workspace.element_size() if workspace_bytes is None else workspace_bytes
    best = qmc_tuning()
    _check(_lib.qmc_tune_integrate(ctypes.byref(problem), n_integrals, _dev(counts), _dev(theta), _dev(target),
                                   _dev(estimate), _dev(grad_theta), _dev(loss), _dev(workspace), wb,
                                   _stream(stream), ctypes.byref(best)), "qmc_tune_integrate")
    return best


def qmc_tune_clear() -> None:
    _check(_lib.qmc_tune_clear(), "qmc_tune_clear")


def qmc_tune_save(path: str) -> None:
    _check(_lib.qmc_tune_save(os.fsencode(path)), "qmc_tune_save")


def qmc_tune_load(path: str) -> int:
    n = c_uint32(0)
    _check(_lib.qmc_tune_load(os.fsencode(path), ctypes.byref(n)), "qmc_tune_load")
    return n.value


def qmc_tune_lookup(problem, n_integrals, with_gradient=False) -> qmc_tuning:
    out = qmc_tuning()
    _check(_lib.qmc_tune_lookup(ctypes.byref(problem), n_integrals, int(bool(with_gradient)), ctypes.byref(out)),
           "qmc_tune_lookup")
    return out


def qmc_graph_begin(stream=None) -> None:
    _check(_lib.qmc_graph_begin(_stream(stream)), "qmc_graph_begin")


def qmc_graph_end(stream=None) -> int:
    g = c_void_p()
    _check(_lib.qmc_graph_end(_stream(stream), ctypes.byref(g)), "qmc_graph_end")
    return g.value


def qmc_graph_launch(graph: int, stream=None) -> None:
    _check(_lib.qmc_graph_launch(graph, _stream(stream)), "qmc_graph_launch")


def qmc_graph_destroy(graph: int) -> None:
    _check(_lib.qmc_graph_destroy(graph), "qmc_graph_destroy")


def qmc_checked_error(reset=False) -> int:
    """The checked build's error bits (synchronises the device); QMCError(6) in the normal build."""
    bits = c_uint32(0)
    _check(_lib.qmc_checked_error(ctypes.byref(bits), int(bool(reset))), "qmc_checked_error")
    return bits.value


def qmc_read_device_error(workspace, stream=None) -> int:
    bits = c_uint32(0)
    _check(_lib.qmc_read_device_error(_dev(workspace), ctypes.byref(bits), _stream(stream)),
           "qmc_read_device_error")
    return bits.value


# ----------------------------------------------------------------- conveniences
def make_problem(source, integrand, s, randomize=0, matrices=None, g=None, seeds=None,
                 seeds_per_integral=False, chunk=0, block=0, max_count=0, with_gradient=False,
                 image_width=0, index_bits=0, partition_log2=0) -> qmc_problem:
    """A qmc_problem holding device pointers of the given tensors; the problem keeps
    references to them so their memory stays valid while it is alive.  Fields as in
    include/qmc.h: for SOURCE_SOBOL, index_bits is the matrices' columns per dimension
    (0 = 32) and partition_log2 = q makes integral p integrate element p mod 2^q of the
    sequence partitioned by the matrices' dimension 0 (which then hold s + 1 dimensions)."""
    p = qmc_problem(source, integrand, s, randomize, _dev(matrices), _dev(g), _dev(seeds),
                    int(bool(seeds_per_integral)), chunk, block, max_count, int(bool(with_gradient)), image_width,
                    index_bits, partition_log2)
    p._tensors = (matrices, g, seeds)
    return p


def alloc_workspace(problem: qmc_problem, n_integrals: int, h_counts=None, device="cuda") -> torch.Tensor:
    nbytes = qmc_integrate_workspace_bytes(problem, n_integrals, h_counts)
    if nbytes == 0:
        raise QMCError(1, "qmc_integrate_workspace_bytes")
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def sobol_points(matrices, count, index_begin=0, scramble=SCRAMBLE_NONE, seeds=None, want_u32=True,
                 want_f32=True, stream=None):
    s = matrices.shape[0]
    dev = matrices.device
    u = torch.empty((count, s), dtype=torch.int32, device=dev) if want_u32 else None
    f = torch.empty((count, s), dtype=torch.float32, device=dev) if want_f32 else None
    qmc_sobol_points(matrices, s, index_begin, count, scramble, seeds, u, f, stream)
    return u, f


def lattice_points(g, count, index_begin=0, shift=None, backward=False, want_u32=True, want_f32=True,
                   stream=None):
    s = g.shape[0]
    dev = g.device
    u = torch.empty((count, s), dtype=torch.int32, device=dev) if want_u32 else None
    f = torch.empty((count, s), dtype=torch.float32, device=dev) if want_f32 else None
    qmc_lattice_points(g, shift, s, index_begin, count, LATTICE_BACKWARD if backward else 0, u, f, stream)
    return u, f
