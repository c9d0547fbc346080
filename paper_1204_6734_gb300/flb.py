"""Python binding of the C ABI in include/flb.h (ctypes; argument marshalling only).

Every function named ``flb_*`` here calls the C entry point of the same name in
``_build/libflb.so``; every step of the method runs in that library's CUDA
kernels. There is no fallback: if the library cannot be loaded the import of
this module's functions raises.

PyTorch is optional and only used as plumbing: a ``torch.cuda.Stream`` (or its
raw handle) may be passed as the stream, and a CUDA ``torch.Tensor`` as the
device workspace.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_OOM, ERR_INVALID_VELOCITY, ERR_NONFINITE, ERR_TIMEOUT, ERR_CUDA, ERR_STATE = (
    -1, -2, -3, -4, -5, -6, -7)
BASIS = {"standard": 0, "local": 1, "lut": 2}
OPT_KERNEL, OPT_PIPELINE_WARPS, OPT_PIPELINE_SAMPLING = 0, 1, 2
KERNEL = {"auto": 0, "generic": 1, "pipelined": 2}
PRECISION = {"fp64": 0, "fp32": 1, "fp16dev": 2}
TILE = {"128x4": 0, "64x8": 1, "128x2": 2, "128x6": 3, "64x12": 4, "mixed": 5}   # tile shapes of the batched kernel
TILE_COUNT = 6


class FlbError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = flb_error_string(code) if _lib is not None else str(code)
        super().__init__(f"{what}: flb error {code} ({msg})" if what else f"flb error {code} ({msg})")
        self.code = code


class flb_params(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32), ("rho0", C.c_double),
                ("ux0", C.c_double), ("uy0", C.c_double), ("kT", C.c_double),
                ("omega", C.c_double * 9), ("basis", C.c_int32), ("precision", C.c_int32),
                ("seed", C.c_uint64), ("replica", C.c_uint32), ("reserved", C.c_uint32)]


class flb_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("reserved", C.c_int32),
                ("steps", C.c_int64), ("n_samples", C.c_int64), ("S1", C.c_double * 9),
                ("S2", C.c_double * 81), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class flb_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("queued", C.c_int64), ("running", C.c_int64),
                ("finishing", C.c_int64), ("completed", C.c_int64), ("pending_results", C.c_int64), ("chunks", C.c_int64),
                ("replica_steps", C.c_int64), ("node_steps", C.c_int64), ("pool_used", C.c_int64),
                ("pool_size", C.c_int64), ("gpu_busy_s", C.c_double), ("clock_s", C.c_double)]


SERVE = {"batched": 0, "per_lattice": 1}

_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libflb.so (building it first if it is missing or stale and nvcc is
    available). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build.stale()):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    L = C.CDLL(path)
    P = C.POINTER(flb_params)
    h = C.c_void_p
    sig = {
        "flb_workspace_bytes": (C.c_size_t, [P]),
        "flb_create": (C.c_int, [P, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(h)]),
        "flb_destroy": (C.c_int, [h]),
        "flb_set_sampling": (C.c_int, [h, C.c_int64, C.c_int64]),
        "flb_reset_statistics": (C.c_int, [h]),
        "flb_step": (C.c_int, [h, C.c_int64]),
        "flb_sync": (C.c_int, [h]),
        "flb_time": (C.c_int, [h, _i64p]),
        "flb_set_time": (C.c_int, [h, C.c_int64]),
        "flb_wait_probe": (C.c_int, [C.c_int64]),
        "flb_set_raw_sums": (C.c_int, [h, _dp, _dp, C.c_int64]),
        "flb_error_location": (C.c_int, [h, _i64p, _i64p]),
        "flb_reset_error": (C.c_int, [h]),
        "flb_correlations": (C.c_int, [h, C.c_int32, _dp, _dp, _dp, _i64p]),
        "flb_raw_sums": (C.c_int, [h, _dp, _dp, _i64p]),
        "flb_conservation": (C.c_int, [h, _dp]),
        "flb_get_populations": (C.c_int, [h, _dp]),
        "flb_state_difference": (C.c_int, [h, h, _dp]),
        "flb_set_structure_sampling": (C.c_int, [h, C.c_int64, C.c_int64]),
        "flb_structure_factors": (C.c_int, [h, _dp, _dp, _dp, _dp, _i64p]),
        "flb_set_populations": (C.c_int, [h, _dp]),
        "flb_run_host": (C.c_int, [P, _dp, C.c_int64, C.c_int64, C.c_int64, _dp, _dp, _dp, _i64p]),
        "flb_noise_draws": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, _u32p, C.c_int32,
                                      C.c_int32, _u32p, _dp]),
        "flb_collide_nodes": (C.c_int, [P, _dp, _u32p, C.c_uint32, C.c_int32, _dp, _i32p]),
        "flb_set_option": (C.c_int, [h, C.c_int32, C.c_int32]),
        "flb_set_slab": (C.c_int, [h, C.c_int32, C.c_int32]),
        "flb_halo_bytes": (C.c_size_t, [h]),
        "flb_halo_pack": (C.c_int, [h, C.c_void_p, C.c_void_p]),
        "flb_halo_unpack": (C.c_int, [h, C.c_void_p, C.c_void_p]),
        "flb_step_noalloc": (C.c_int, [P, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, _dp, _dp,
                                       C.c_void_p]),
        "flb_batch_open": (C.c_int, [C.c_int32, C.c_int32, C.c_size_t, C.c_void_p, C.POINTER(h)]),
        "flb_batch_replica_bytes": (C.c_size_t, [P]),
        "flb_batch_add": (C.c_int, [h, P, C.c_int64, _i32p]),
        "flb_batch_remove": (C.c_int, [h, C.c_int32]),
        "flb_batch_create": (C.c_int, [P, C.c_int32, C.c_void_p, C.POINTER(h)]),
        "flb_batch_workspace_bytes": (C.c_size_t, [P, C.c_int32]),
        "flb_batch_destroy": (C.c_int, [h]),
        "flb_batch_set_sampling": (C.c_int, [h, C.c_int32, C.c_int64, C.c_int64]),
        "flb_batch_step": (C.c_int, [h, C.c_int64]),
        "flb_batch_set_graph": (C.c_int, [h, C.c_int32]),
        "flb_batch_set_tile": (C.c_int, [h, C.c_int32]),
        "flb_batch_get_tile": (C.c_int, [h, _i32p]),
        "flb_batch_autotune": (C.c_int, [h, C.c_int32, _i32p, _dp]),
        "flb_batch_sync": (C.c_int, [h]),
        "flb_batch_status": (C.c_int, [h, C.c_int32]),
        "flb_batch_time": (C.c_int, [h, _i64p]),
        "flb_batch_replica_time": (C.c_int, [h, C.c_int32, _i64p]),
        "flb_batch_info": (C.c_int, [h, _i32p, _i64p, C.POINTER(C.c_size_t),
                                     C.POINTER(C.c_size_t)]),
        "flb_batch_raw_sums": (C.c_int, [h, C.c_int32, _dp, _dp, _i64p]),
        "flb_batch_correlations": (C.c_int, [h, C.c_int32, _i32p, C.c_int32, _dp, _dp, _dp, _i64p]),
        "flb_batch_get_populations": (C.c_int, [h, C.c_int32, _dp]),
        "flb_batch_set_populations": (C.c_int, [h, C.c_int32, _dp]),
        "flb_server_create": (C.c_int, [C.c_int32, C.c_int32, C.c_size_t, C.c_int32, C.c_int32,
                                        C.c_void_p, C.POINTER(h)]),
        "flb_server_destroy": (C.c_int, [h]),
        "flb_server_submit": (C.c_int, [h, P, C.c_int64, C.c_int64, C.c_int64, _i64p]),
        "flb_server_poll": (C.c_int, [h, C.c_int32, C.c_int32, C.POINTER(flb_result), _i32p]),
        "flb_server_stats": (C.c_int, [h, C.POINTER(flb_serve_stats)]),
        "flb_server_set_tile": (C.c_int, [h, C.c_int32]),
        "flb_error_string": (C.c_char_p, [C.c_int]),
        "flb_version": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points this binding expects."""
    return ["flb_workspace_bytes", "flb_create", "flb_destroy", "flb_set_sampling",
            "flb_reset_statistics", "flb_step", "flb_sync", "flb_time", "flb_error_location",
            "flb_reset_error", "flb_correlations", "flb_raw_sums", "flb_conservation",
            "flb_get_populations", "flb_set_populations", "flb_run_host", "flb_noise_draws",
            "flb_collide_nodes", "flb_set_option", "flb_step_noalloc", "flb_error_string",
            "flb_set_slab", "flb_halo_bytes", "flb_halo_pack", "flb_halo_unpack",
            "flb_version", "flb_state_difference", "flb_batch_open", "flb_batch_replica_bytes", "flb_batch_add",
            "flb_batch_remove", "flb_batch_create", "flb_batch_workspace_bytes",
            "flb_batch_destroy", "flb_batch_set_sampling", "flb_batch_step",
            "flb_batch_set_graph", "flb_batch_set_tile", "flb_batch_get_tile",
            "flb_batch_autotune", "flb_batch_sync", "flb_batch_status", "flb_batch_time",
            "flb_batch_replica_time", "flb_batch_info", "flb_batch_raw_sums",
            "flb_batch_get_populations", "flb_batch_set_populations", "flb_server_create",
            "flb_server_destroy", "flb_server_submit", "flb_server_poll", "flb_server_stats",
            "flb_server_set_tile", "flb_set_structure_sampling", "flb_structure_factors",
            "flb_batch_correlations", "flb_set_time", "flb_set_raw_sums", "flb_wait_probe"]


def _check(rc: int, what: str):
    if rc != OK:
        raise FlbError(rc, what)


def make_params(p) -> flb_params:
    """flb_params from any object with Lx, Ly, rho0, ux0, uy0, kT, omega, basis,
    precision, seed and (optionally) replica attributes."""
    s = flb_params()
    s.Lx, s.Ly = int(p.Lx), int(p.Ly)
    s.rho0, s.ux0, s.uy0, s.kT = float(p.rho0), float(p.ux0), float(p.uy0), float(p.kT)
    for a, v in enumerate(p.omega):
        s.omega[a] = float(v)
    s.basis = BASIS[p.basis] if isinstance(p.basis, str) else int(p.basis)
    prec = getattr(p, "precision", "fp32")
    s.precision = PRECISION[prec] if isinstance(prec, str) else int(prec)
    s.seed = int(p.seed) & 0xFFFFFFFFFFFFFFFF
    s.replica = int(getattr(p, "replica", 0))
    s.reserved = 0
    return s


def _ptr(a, ctype=C.c_double):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


# ---------------------------------------------------------------------------
# Same-name wrappers of the C entry points
# ---------------------------------------------------------------------------

def flb_error_string(code: int) -> str:
    return load().flb_error_string(code).decode()


def flb_version() -> int:
    return load().flb_version()


def flb_workspace_bytes(p) -> int:
    s = make_params(p)
    return int(load().flb_workspace_bytes(C.byref(s)))


def flb_create(p, workspace=None, stream=None):
    s = make_params(p)
    h = C.c_void_p()
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr = int(workspace.data_ptr())
        ws_bytes = int(workspace.numel() * workspace.element_size())
    _check(load().flb_create(C.byref(s), ws_ptr, ws_bytes, _stream_handle(stream), C.byref(h)),
           "flb_create")
    return h


def flb_destroy(h) -> None:
    _check(load().flb_destroy(h), "flb_destroy")


def flb_set_sampling(h, warmup: int, every: int) -> None:
    _check(load().flb_set_sampling(h, int(warmup), int(every)), "flb_set_sampling")


def flb_reset_statistics(h) -> None:
    _check(load().flb_reset_statistics(h), "flb_reset_statistics")


def flb_step(h, n: int) -> None:
    _check(load().flb_step(h, int(n)), "flb_step")


def flb_sync(h) -> None:
    _check(load().flb_sync(h), "flb_sync")


def flb_wait_probe(limit_cycles: int) -> int:
    """Return code of a bounded wait on a barrier nothing completes
    (FLB_ERR_TIMEOUT expected)."""
    return int(load().flb_wait_probe(int(limit_cycles)))


def flb_set_time(h, t: int) -> None:
    _check(load().flb_set_time(h, int(t)), "flb_set_time")


def flb_set_raw_sums(h, S1, S2, n_samples: int) -> None:
    S1 = np.ascontiguousarray(S1, dtype=np.float64)
    S2 = np.ascontiguousarray(S2, dtype=np.float64)
    assert S1.size == 9 and S2.size == 81
    _check(load().flb_set_raw_sums(h, _ptr(S1), _ptr(S2), int(n_samples)), "flb_set_raw_sums")


def flb_time(h) -> int:
    t = C.c_int64()
    _check(load().flb_time(h, C.byref(t)), "flb_time")
    return t.value


def flb_set_option(h, option: int, value: int) -> None:
    _check(load().flb_set_option(h, int(option), int(value)), "flb_set_option")


def flb_error_location(h):
    n, s = C.c_int64(), C.c_int64()
    _check(load().flb_error_location(h, C.byref(n), C.byref(s)), "flb_error_location")
    return n.value, s.value


def flb_reset_error(h) -> None:
    _check(load().flb_reset_error(h), "flb_reset_error")


def flb_correlations(h, measure_basis="local"):
    Cff, CMM, mean = np.zeros((9, 9)), np.zeros((9, 9)), np.zeros(9)
    n = C.c_int64()
    mb = BASIS[measure_basis] if isinstance(measure_basis, str) else int(measure_basis)
    _check(load().flb_correlations(h, mb, _ptr(Cff), _ptr(CMM), _ptr(mean), C.byref(n)),
           "flb_correlations")
    return Cff, CMM, mean, n.value


def flb_raw_sums(h):
    S1, S2 = np.zeros(9), np.zeros((9, 9))
    n = C.c_int64()
    _check(load().flb_raw_sums(h, _ptr(S1), _ptr(S2), C.byref(n)), "flb_raw_sums")
    return S1, S2, n.value


def flb_conservation(h):
    out = np.zeros(3)
    _check(load().flb_conservation(h, _ptr(out)), "flb_conservation")
    return out


def flb_state_difference(a, b):
    """(max |f_a - f_b|, RMS of f_a - f_b, max |f_b|) of two lattices' states."""
    out = np.zeros(3)
    _check(load().flb_state_difference(a, b, _ptr(out)), "flb_state_difference")
    return tuple(out)


def flb_set_structure_sampling(h, warmup: int, every: int) -> None:
    _check(load().flb_set_structure_sampling(h, int(warmup), int(every)),
           "flb_set_structure_sampling")


def flb_structure_factors(h, Lx: int, Ly: int):
    """(S_rho, S_jx, R, n_samples): S_k(rho), S_k(j_x) and the complex
    R_k(j_x, j_y), each (Ly, Lx) indexed [m_y, m_x]."""
    Sr, Sx = np.empty((Ly, Lx)), np.empty((Ly, Lx))
    Rr, Ri = np.empty((Ly, Lx)), np.empty((Ly, Lx))
    n = C.c_int64()
    _check(load().flb_structure_factors(h, _ptr(Sr), _ptr(Sx), _ptr(Rr), _ptr(Ri), C.byref(n)),
           "flb_structure_factors")
    return Sr, Sx, Rr + 1j * Ri, n.value


def flb_get_populations(h, Lx: int, Ly: int, out=None):
    if out is None:
        out = np.empty((9, Ly, Lx))
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 9 * Lx * Ly
    _check(load().flb_get_populations(h, _ptr(out)), "flb_get_populations")
    return out


def flb_set_populations(h, f) -> None:
    a = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().flb_set_populations(h, _ptr(a)), "flb_set_populations")


def flb_run_host(p, f_in, nsteps, warmup=0, every=0, f_out=None):
    s = make_params(p)
    fi = None if f_in is None else np.ascontiguousarray(f_in, dtype=np.float64)
    S1, S2 = np.zeros(9), np.zeros((9, 9))
    n = C.c_int64()
    _check(load().flb_run_host(C.byref(s), _ptr(fi), int(nsteps), int(warmup), int(every),
                               _ptr(f_out), _ptr(S1), _ptr(S2), C.byref(n)), "flb_run_host")
    return S1, S2, n.value


def flb_noise_draws(seed, replica, step, nodes, precision="fp64"):
    nd = np.ascontiguousarray(nodes, dtype=np.uint32)
    n = nd.size
    fields = np.zeros((n, 6), dtype=np.uint32)
    normals = np.zeros((n, 6))
    pr = PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(load().flb_noise_draws(int(seed) & 0xFFFFFFFFFFFFFFFF, int(replica), int(step),
                                  _ptr(nd, C.c_uint32), n, pr, _ptr(fields, C.c_uint32),
                                  _ptr(normals)), "flb_noise_draws")
    return fields, normals


def flb_collide_nodes(p, g, node_ids, step):
    s = make_params(p)
    gg = np.ascontiguousarray(g, dtype=np.float64).reshape(-1, 9)
    ids = np.ascontiguousarray(node_ids, dtype=np.uint32)
    n = gg.shape[0]
    out = np.zeros((n, 9))
    st = np.zeros(n, dtype=np.int32)
    _check(load().flb_collide_nodes(C.byref(s), _ptr(gg), _ptr(ids, C.c_uint32), int(step), n,
                                    _ptr(out), _ptr(st, C.c_int32)), "flb_collide_nodes")
    return out, st


def flb_step_noalloc(p, dev_f, dev_work, t0, nsteps, stream=None):
    """FP64 steps on caller-owned device buffers (CUDA tensors or raw device
    pointers) without any device allocation; returns the sampled sums
    (S1[9], S2[9,9]) of this call."""
    s = make_params(p)
    S1, S2 = np.zeros(9), np.zeros((9, 9))
    f = dev_f if isinstance(dev_f, int) else int(dev_f.data_ptr())
    w = dev_work if isinstance(dev_work, int) else int(dev_work.data_ptr())
    _check(load().flb_step_noalloc(C.byref(s), f, w, int(t0), int(nsteps), _ptr(S1), _ptr(S2),
                                   _stream_handle(stream)), "flb_step_noalloc")
    return S1, S2


def flb_set_slab(h, Ly_total: int, y0: int):
    _check(load().flb_set_slab(h, int(Ly_total), int(y0)), "flb_set_slab")


def flb_halo_bytes(h) -> int:
    return int(load().flb_halo_bytes(h))


def _dev_ptr(x):
    return x if isinstance(x, int) else int(x.data_ptr())


def flb_halo_pack(h, lo, hi):
    """lo, hi: device buffers (CUDA tensors or raw pointers) of flb_halo_bytes(h)."""
    _check(load().flb_halo_pack(h, _dev_ptr(lo), _dev_ptr(hi)), "flb_halo_pack")


def flb_halo_unpack(h, lo, hi):
    _check(load().flb_halo_unpack(h, _dev_ptr(lo), _dev_ptr(hi)), "flb_halo_unpack")


def _param_array(ps):
    arr = (flb_params * len(ps))()
    for k, p in enumerate(ps):
        arr[k] = make_params(p)
    return arr


def flb_batch_open(basis, max_replicas: int, pool_bytes: int, stream=None):
    b = C.c_void_p()
    bs = BASIS[basis] if isinstance(basis, str) else int(basis)
    _check(load().flb_batch_open(bs, int(max_replicas), int(pool_bytes), _stream_handle(stream),
                                 C.byref(b)), "flb_batch_open")
    return b


def flb_batch_replica_bytes(p) -> int:
    s = make_params(p)
    return int(load().flb_batch_replica_bytes(C.byref(s)))


def flb_batch_add(b, p, nsteps: int = 0) -> int:
    s = make_params(p)
    slot = C.c_int32()
    _check(load().flb_batch_add(b, C.byref(s), int(nsteps), C.byref(slot)), "flb_batch_add")
    return slot.value


def flb_batch_remove(b, slot: int) -> None:
    _check(load().flb_batch_remove(b, int(slot)), "flb_batch_remove")


def flb_batch_create(ps, stream=None):
    arr = _param_array(ps)
    b = C.c_void_p()
    _check(load().flb_batch_create(arr, len(ps), _stream_handle(stream), C.byref(b)),
           "flb_batch_create")
    return b


def flb_batch_workspace_bytes(ps) -> int:
    arr = _param_array(ps)
    return int(load().flb_batch_workspace_bytes(arr, len(ps)))


def flb_batch_destroy(b) -> None:
    _check(load().flb_batch_destroy(b), "flb_batch_destroy")


def flb_batch_set_sampling(b, slot: int, warmup: int, every: int) -> None:
    _check(load().flb_batch_set_sampling(b, int(slot), int(warmup), int(every)),
           "flb_batch_set_sampling")


def flb_batch_step(b, n: int) -> None:
    _check(load().flb_batch_step(b, int(n)), "flb_batch_step")


def flb_batch_set_graph(b, steps: int) -> None:
    _check(load().flb_batch_set_graph(b, int(steps)), "flb_batch_set_graph")


def flb_batch_set_tile(b, tile) -> None:
    v = TILE[tile] if isinstance(tile, str) else int(tile)
    _check(load().flb_batch_set_tile(b, v), "flb_batch_set_tile")


def flb_batch_get_tile(b) -> int:
    v = C.c_int32()
    _check(load().flb_batch_get_tile(b, C.byref(v)), "flb_batch_get_tile")
    return v.value


def flb_batch_autotune(b, trial_steps: int):
    """Returns (chosen tile index, ms per step of every tile shape)."""
    tile = C.c_int32()
    ms = np.zeros(TILE_COUNT)
    _check(load().flb_batch_autotune(b, int(trial_steps), C.byref(tile), _ptr(ms)),
           "flb_batch_autotune")
    return tile.value, ms


def flb_batch_sync(b) -> None:
    _check(load().flb_batch_sync(b), "flb_batch_sync")


def flb_batch_status(b, slot: int) -> int:
    """FLB status code of one replica (0 = OK); raises only for a bad slot."""
    rc = load().flb_batch_status(b, int(slot))
    if rc == ERR_ARG:
        raise FlbError(rc, "flb_batch_status")
    return rc


def flb_batch_time(b) -> int:
    t = C.c_int64()
    _check(load().flb_batch_time(b, C.byref(t)), "flb_batch_time")
    return t.value


def flb_batch_replica_time(b, slot: int) -> int:
    t = C.c_int64()
    _check(load().flb_batch_replica_time(b, int(slot), C.byref(t)), "flb_batch_replica_time")
    return t.value


def flb_batch_info(b):
    """(live replicas, tiles in the current shape, pool bytes used, pool size)."""
    n, t = C.c_int32(), C.c_int64()
    used, size = C.c_size_t(), C.c_size_t()
    _check(load().flb_batch_info(b, C.byref(n), C.byref(t), C.byref(used), C.byref(size)),
           "flb_batch_info")
    return n.value, t.value, used.value, size.value


def flb_batch_raw_sums(b, slot: int):
    S1, S2 = np.zeros(9), np.zeros((9, 9))
    n = C.c_int64()
    _check(load().flb_batch_raw_sums(b, int(slot), _ptr(S1), _ptr(S2), C.byref(n)),
           "flb_batch_raw_sums")
    return S1, S2, n.value


def flb_batch_correlations(b, slots, measure_basis="local"):
    """(Cff, CMM, mean, n) pooled over the given replicas (same rho0, u0)."""
    sl = np.ascontiguousarray(np.asarray(slots, dtype=np.int32))
    Cff, CMM, mean = np.zeros((9, 9)), np.zeros((9, 9)), np.zeros(9)
    n = C.c_int64()
    mb = BASIS[measure_basis] if isinstance(measure_basis, str) else int(measure_basis)
    _check(load().flb_batch_correlations(b, len(sl), sl.ctypes.data_as(_i32p), mb, _ptr(Cff), _ptr(CMM),
                                         _ptr(mean), C.byref(n)), "flb_batch_correlations")
    return Cff, CMM, mean, n.value


def flb_batch_get_populations(b, slot: int, Lx: int, Ly: int, out=None):
    if out is None:
        out = np.empty((9, Ly, Lx))
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 9 * Lx * Ly
    _check(load().flb_batch_get_populations(b, int(slot), _ptr(out)), "flb_batch_get_populations")
    return out


def flb_batch_set_populations(b, slot: int, f) -> None:
    a = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().flb_batch_set_populations(b, int(slot), _ptr(a)), "flb_batch_set_populations")


def flb_server_create(mode, basis, pool_bytes: int, max_slots: int, chunk_steps: int, stream=None):
    s = C.c_void_p()
    m = SERVE[mode] if isinstance(mode, str) else int(mode)
    bs = BASIS[basis] if isinstance(basis, str) else int(basis)
    _check(load().flb_server_create(m, bs, int(pool_bytes), int(max_slots), int(chunk_steps),
                                    _stream_handle(stream), C.byref(s)), "flb_server_create")
    return s


def flb_server_destroy(s) -> None:
    _check(load().flb_server_destroy(s), "flb_server_destroy")


def flb_server_submit(s, p, nsteps: int, warmup: int = 0, every: int = 0) -> int:
    q = make_params(p)
    rid = C.c_int64()
    _check(load().flb_server_submit(s, C.byref(q), int(nsteps), int(warmup), int(every),
                                    C.byref(rid)), "flb_server_submit")
    return rid.value


def flb_server_poll(s, wait: bool = False, max_results: int = 64):
    """List of finished requests as dicts (id, status, steps, n_samples, S1,
    S2, t_submit, t_admit, t_done)."""
    buf = (flb_result * max_results)()
    n = C.c_int32()
    _check(load().flb_server_poll(s, 1 if wait else 0, max_results, buf, C.byref(n)),
           "flb_server_poll")
    out = []
    for k in range(n.value):
        r = buf[k]
        out.append({"id": r.id, "status": r.status, "steps": r.steps, "n_samples": r.n_samples,
                    "S1": np.array(r.S1[:]), "S2": np.array(r.S2[:]).reshape(9, 9),
                    "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done})
    return out


def flb_server_set_tile(s, tile) -> None:
    v = TILE[tile] if isinstance(tile, str) else int(tile)
    _check(load().flb_server_set_tile(s, v), "flb_server_set_tile")


def flb_server_stats(s) -> dict:
    st = flb_serve_stats()
    _check(load().flb_server_stats(s, C.byref(st)), "flb_server_stats")
    return {name: getattr(st, name) for name, _ in flb_serve_stats._fields_}


# ---------------------------------------------------------------------------
# Convenience object
# ---------------------------------------------------------------------------

class Lattice:
    """One periodic lattice on the GPU (owns an flb_lattice handle)."""

    def __init__(self, p, workspace=None, stream=None, kernel=None, pipeline_warps=None,
                 pipeline_sampling=None):
        self.p = p
        self.h = flb_create(p, workspace, stream)
        if kernel is not None:
            flb_set_option(self.h, OPT_KERNEL, KERNEL[kernel] if isinstance(kernel, str) else kernel)
        if pipeline_sampling is not None:
            flb_set_option(self.h, OPT_PIPELINE_SAMPLING, pipeline_sampling)
        if pipeline_warps is not None:
            flb_set_option(self.h, OPT_PIPELINE_WARPS, pipeline_warps)

    def close(self):
        if self.h is not None:
            flb_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_sampling(self, warmup, every):
        flb_set_sampling(self.h, warmup, every)

    def step(self, n):
        flb_step(self.h, n)
        return self

    def sync(self):
        flb_sync(self.h)

    @property
    def t(self):
        return flb_time(self.h)

    def populations(self):
        return flb_get_populations(self.h, self.p.Lx, self.p.Ly)

    def set_populations(self, f):
        flb_set_populations(self.h, f)

    def correlations(self, measure_basis="local"):
        return flb_correlations(self.h, measure_basis)

    def raw_sums(self):
        return flb_raw_sums(self.h)

    def checkpoint(self):
        """(populations, t, (S1, S2, n)): what resume() needs to continue."""
        return self.populations(), self.t, self.raw_sums()

    def resume(self, state, warmup, every):
        """Continue a checkpointed run on this handle (same parameters):
        the sampling schedule, the sums, the time and the state."""
        f, t, (S1, S2, n) = state
        self.set_sampling(warmup, every)
        flb_set_raw_sums(self.h, S1, S2, n)
        flb_set_time(self.h, t)
        self.set_populations(f)

    def set_structure_sampling(self, warmup, every):
        flb_set_structure_sampling(self.h, warmup, every)

    def structure_factors(self):
        return flb_structure_factors(self.h, self.p.Lx, self.p.Ly)

    def conservation(self):
        return flb_conservation(self.h)


class Batch:
    """Many FP32 lattices stepped by one launch per step (owns an flb_batch).

    ``Batch(params_list)`` adds the given lattices as slots 0..n-1 with no step
    limit; ``Batch.open(basis, max_replicas, pool_bytes)`` starts empty, for
    replicas that join and leave (``add`` / ``remove``)."""

    def __init__(self, ps=None, stream=None, graph_steps=0, tile=None, _handle=None):
        self.params = {}
        if _handle is not None:
            self.h = _handle
        else:
            self.h = flb_batch_create(list(ps), stream)
            self.params = {k: p for k, p in enumerate(ps)}
        if graph_steps:
            flb_batch_set_graph(self.h, graph_steps)
        if tile is not None:
            flb_batch_set_tile(self.h, tile)

    @classmethod
    def open(cls, basis, max_replicas, pool_bytes, stream=None, graph_steps=0):
        return cls(stream=stream, graph_steps=graph_steps,
                   _handle=flb_batch_open(basis, max_replicas, pool_bytes, stream))

    def add(self, p, nsteps=0):
        slot = flb_batch_add(self.h, p, nsteps)
        self.params[slot] = p
        return slot

    def remove(self, slot):
        flb_batch_remove(self.h, slot)
        self.params.pop(slot, None)

    def close(self):
        if getattr(self, "h", None) is not None:
            flb_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_sampling(self, warmup, every, slot=-1):
        flb_batch_set_sampling(self.h, slot, warmup, every)

    def step(self, n):
        flb_batch_step(self.h, n)
        return self

    def sync(self):
        flb_batch_sync(self.h)

    def status(self, slot):
        return flb_batch_status(self.h, slot)

    def set_tile(self, tile):
        flb_batch_set_tile(self.h, tile)

    @property
    def tile(self):
        return flb_batch_get_tile(self.h)

    def autotune(self, trial_steps=20):
        return flb_batch_autotune(self.h, trial_steps)

    def set_graph(self, steps):
        flb_batch_set_graph(self.h, steps)

    @property
    def t(self):
        return flb_batch_time(self.h)

    def replica_time(self, slot):
        return flb_batch_replica_time(self.h, slot)

    def info(self):
        return flb_batch_info(self.h)

    def raw_sums(self, slot):
        return flb_batch_raw_sums(self.h, slot)

    def correlations(self, slots, measure_basis="local"):
        return flb_batch_correlations(self.h, slots, measure_basis)

    def populations(self, slot):
        p = self.params[slot]
        return flb_batch_get_populations(self.h, slot, p.Lx, p.Ly)

    def set_populations(self, slot, f):
        flb_batch_set_populations(self.h, slot, f)


class Server:
    """Continuous-batching request server (owns an flb_server)."""

    def __init__(self, basis="local", pool_bytes=1 << 30, max_slots=256, chunk_steps=16,
                 mode="batched", stream=None):
        self.h = flb_server_create(mode, basis, pool_bytes, max_slots, chunk_steps, stream)

    def submit(self, p, nsteps, warmup=0, every=0):
        return flb_server_submit(self.h, p, nsteps, warmup, every)

    def poll(self, wait=False, max_results=64):
        return flb_server_poll(self.h, wait, max_results)

    def stats(self):
        return flb_server_stats(self.h)

    def set_tile(self, tile):
        flb_server_set_tile(self.h, tile)

    def drain(self):
        """Poll (blocking) until every submitted request has a result."""
        out = []
        while True:
            st = self.stats()
            if st["completed"] == st["submitted"] and st["pending_results"] == 0:
                return out
            out += self.poll(wait=True)

    def close(self):
        if getattr(self, "h", None) is not None:
            flb_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
