"""Python binding of libttn (include/ttn.h): argument marshalling only.

Every function has the name of the C entry point it calls and converts
NumPy arrays to the C layouts; all computation happens in the CUDA library.
If ``libttn.so`` has not been built this module raises on import -- there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libttn.so")

TTN_OK, TTN_E_INVALID, TTN_E_OOM, TTN_E_CUDA, TTN_E_NOCONV, TTN_E_TIMEOUT, TTN_E_STATE = range(7)
TTN_FP64, TTN_MIXED = 0, 1
STATUS_NAMES = {0: "TTN_OK", 1: "TTN_E_INVALID", 2: "TTN_E_OOM", 3: "TTN_E_CUDA",
                4: "TTN_E_NOCONV", 5: "TTN_E_TIMEOUT", 6: "TTN_E_STATE"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2503_15460_gb300.build.build()")
_lib = C.CDLL(LIB_PATH)


class ttn_step_opts(C.Structure):
    _fields_ = [("krylov_tol", C.c_double), ("krylov_maxdim", C.c_int),
                ("eps_spawn", C.c_double), ("chi_max", C.c_int), ("expand", C.c_int),
                ("qr_rank_tol", C.c_double)]


class ttn_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_slots", C.c_int), ("slice_ms", C.c_double),
                ("use_graph", C.c_int)]


class ttn_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queued", C.c_int64), ("running", C.c_int64), ("steps", C.c_int64),
                ("launches", C.c_int64), ("peak_running", C.c_int64), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("p50_step_ms", C.c_double), ("p99_step_ms", C.c_double),
                ("n_latencies", C.c_int64)]


_P = C.c_void_p
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_C128 = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_F64 = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")

_sig = {
    "ttn_create": ([C.c_int, _I32, _I32, _I32, C.c_int, C.POINTER(_P)], C.c_int),
    "ttn_create_host": ([C.c_int, _I32, _I32, _I32, C.c_int, C.POINTER(_P)], C.c_int),
    "ttn_materialize": ([_P], C.c_int),
    "ttn_evict": ([_P], C.c_int),
    "ttn_footprint": ([_P, C.POINTER(C.c_size_t)], C.c_int),
    "ttn_set_state": ([_P, _C128, _I64], C.c_int),
    "ttn_set_product_state": ([_P, _C128, _I64], C.c_int),
    "ttn_set_sop_hamiltonian": ([_P, C.c_int, _C128, _I32, _I32, _C128, _I64, C.c_int], C.c_int),
    "ttn_set_multiset_hamiltonian": ([_P, C.c_int, C.c_int, _C128, _I32, _I32, _C128, _I64, _I32, _I32, C.c_int],
                                     C.c_int),
    "ttn_set_multiset_state": ([_P, C.c_int, _C128, _I64], C.c_int),
    "ttn_get_multiset_state": ([_P, C.c_int, _C128, _I64], C.c_int),
    "ttn_set_populations": ([_P, _F64], C.c_int),
    "ttn_n_sets": ([_P, C.POINTER(C.c_int)], C.c_int),
    "ttn_step": ([_P, C.c_double, C.c_int, C.POINTER(ttn_step_opts)], C.c_int),
    "ttn_step_batch": ([C.POINTER(_P), C.c_int, C.c_double, C.c_int, C.POINTER(ttn_step_opts)], C.c_int),
    "ttn_ground_state": ([_P, C.c_int, _F64], C.c_int),
    "ttn_set_coefficients": ([_P, C.c_int, _C128], C.c_int),
    "ttn_save": ([_P, C.c_void_p, C.POINTER(C.c_size_t)], C.c_int),
    "ttn_load": ([_P, C.c_void_p, C.c_size_t], C.c_int),
    "ttn_reduced_density": ([_P, C.c_int, _C128], C.c_int),
    "ttn_expect": ([_P, C.c_int, _I32, _C128, _I64, _C128], C.c_int),
    "ttn_norm_energy": ([_P, C.POINTER(C.c_double), _C128], C.c_int),
    "ttn_vacuum_projection": ([_P, C.c_int, _C128], C.c_int),
    "ttn_get_state": ([_P, _C128, _I64], C.c_int),
    "ttn_bond_dims": ([_P, _I32], C.c_int),
    "ttn_tree": ([_P, C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "ttn_set_stream": ([_P, _P], C.c_int),
    "ttn_set_device": ([C.c_int], C.c_int),
    "ttn_set_cluster": ([_P, C.c_int], C.c_int),
    "ttn_pipe_peaks": ([_P, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "ttn_autotune": ([_P, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "ttn_set_tuning": ([_P, C.c_int, np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")], C.c_int),
    "ttn_operator_dims": ([_P, _I32], C.c_int),
    "ttn_tuning": ([_P, C.POINTER(C.c_int), np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS"),
                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)], C.c_int),
    "ttn_mode_product_c64": ([_P, C.c_int64, C.c_int, C.c_int64, _P, _P, _P, C.c_double, C.c_double, C.c_int,
                              C.c_int], C.c_int),
    "ttn_get_cluster": ([_P, C.POINTER(C.c_int)], C.c_int),
    "ttn_heff_apply": ([_P, C.c_int, _I32, C.c_int, _C128, _I32, C.c_int, C.POINTER(_P), _P, _P], C.c_int),
    "ttn_heff_apply_noalloc": ([_P, C.c_int, _I32, C.c_int, _C128, _I32, C.c_int, C.POINTER(_P), _P, _P], C.c_int),
    "ttn_op_cycles": ([_P, np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")], C.c_int),
    "ttn_step_stats": ([_P, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                        np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS"), C.c_int,
                        C.POINTER(C.c_int)], C.c_int),
    "ttn_device_bytes": ([_P, C.POINTER(C.c_size_t)], C.c_int),
    "ttn_flop_counts": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "ttn_last_error": ([_P], C.c_char_p),
    "ttn_destroy": ([_P], None),
    "ttn_server_create": ([C.c_int, C.POINTER(ttn_server_opts), C.POINTER(_P)], C.c_int),
    "ttn_server_submit": ([_P, _P, C.c_double, C.c_int, C.POINTER(ttn_step_opts), C.POINTER(C.c_int64)], C.c_int),
    "ttn_server_pump": ([_P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "ttn_server_drain": ([_P], C.c_int),
    "ttn_server_poll": ([_P, C.c_int, _I64, _I32, C.POINTER(C.c_int)], C.c_int),
    "ttn_server_get_stats": ([_P, C.POINTER(ttn_server_stats)], C.c_int),
    "ttn_server_latencies": ([_P, _F64, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "ttn_server_last_error": ([_P], C.c_char_p),
    "ttn_server_destroy": ([_P], None),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_sig)


class TTNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st, ctx):
    if st != TTN_OK:
        raise TTNError(st, ttn_last_error(ctx))


def ttn_last_error(ctx) -> str:
    m = _lib.ttn_last_error(ctx)
    return m.decode() if m else ""


def ttn_create(parent, phys_dim, bond_dim, precision=TTN_FP64):
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    phys = np.ascontiguousarray(phys_dim, dtype=np.int32)
    bond = np.ascontiguousarray(bond_dim, dtype=np.int32)
    h = _P()
    st = _lib.ttn_create(len(parent), parent, phys, bond, int(precision), C.byref(h))
    _check(st, None)
    return h


def ttn_create_host(parent, phys_dim, bond_dim, precision=TTN_FP64):
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    phys = np.ascontiguousarray(phys_dim, dtype=np.int32)
    bond = np.ascontiguousarray(bond_dim, dtype=np.int32)
    h = _P()
    st = _lib.ttn_create_host(len(parent), parent, phys, bond, int(precision), C.byref(h))
    _check(st, None)
    return h


def ttn_materialize(ctx):
    _check(_lib.ttn_materialize(ctx), ctx)


def ttn_evict(ctx):
    _check(_lib.ttn_evict(ctx), ctx)


def ttn_footprint(ctx):
    n = C.c_size_t(0)
    _check(_lib.ttn_footprint(ctx, C.byref(n)), ctx)
    return n.value


def _flatten(tensors):
    offs = np.zeros(len(tensors) + 1, dtype=np.int64)
    for i, a in enumerate(tensors):
        offs[i + 1] = offs[i] + np.asarray(a).size
    flat = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.complex128).ravel() for a in tensors]))
    return flat, offs


def ttn_set_state(ctx, tensors):
    flat, offs = _flatten(tensors)
    _check(_lib.ttn_set_state(ctx, flat, offs), ctx)


def ttn_set_product_state(ctx, leaf_vecs: dict, n_nodes: int):
    vecs, offs, o = [], np.zeros(n_nodes, dtype=np.int64), 0
    for z in range(n_nodes):
        offs[z] = o
        if z in leaf_vecs:
            v = np.asarray(leaf_vecs[z], dtype=np.complex128).ravel()
            vecs.append(v); o += v.size
    flat = np.ascontiguousarray(np.concatenate(vecs)) if vecs else np.zeros(1, np.complex128)
    _check(_lib.ttn_set_product_state(ctx, flat, offs), ctx)


def ttn_set_sop_hamiltonian(ctx, coeff, term_ptr, factor_leaf, factor_mats, factor_mat_off, hermitian):
    coeff = np.ascontiguousarray(coeff, dtype=np.complex128)
    term_ptr = np.ascontiguousarray(term_ptr, dtype=np.int32)
    factor_leaf = np.ascontiguousarray(factor_leaf, dtype=np.int32)
    if factor_leaf.size == 0:
        factor_leaf = np.zeros(1, np.int32)
    mats = np.ascontiguousarray(factor_mats, dtype=np.complex128)
    if mats.size == 0:
        mats = np.zeros(1, np.complex128)
    off = np.ascontiguousarray(factor_mat_off, dtype=np.int64)
    if off.size == 0:
        off = np.zeros(1, np.int64)
    _check(_lib.ttn_set_sop_hamiltonian(ctx, len(coeff), coeff, term_ptr, factor_leaf, mats, off,
                                        int(bool(hermitian))), ctx)


def ttn_set_multiset_hamiltonian(ctx, n_sets, coeff, term_ptr, factor_leaf, factor_mats, factor_mat_off, bra, ket,
                                 hermitian):
    coeff = np.ascontiguousarray(coeff, dtype=np.complex128)
    term_ptr = np.ascontiguousarray(term_ptr, dtype=np.int32)
    factor_leaf = np.ascontiguousarray(factor_leaf, dtype=np.int32)
    if factor_leaf.size == 0:
        factor_leaf = np.zeros(1, np.int32)
    mats = np.ascontiguousarray(factor_mats, dtype=np.complex128)
    if mats.size == 0:
        mats = np.zeros(1, np.complex128)
    off = np.ascontiguousarray(factor_mat_off, dtype=np.int64)
    if off.size == 0:
        off = np.zeros(1, np.int64)
    bra = np.ascontiguousarray(bra, dtype=np.int32)
    ket = np.ascontiguousarray(ket, dtype=np.int32)
    _check(_lib.ttn_set_multiset_hamiltonian(ctx, int(n_sets), len(coeff), coeff, term_ptr, factor_leaf, mats, off,
                                             bra, ket, int(bool(hermitian))), ctx)


def ttn_set_multiset_state(ctx, tensor_sets):
    """tensor_sets[alpha][z]: the tensor of set alpha at node z."""
    flat, offs = _flatten([np.asarray(a, dtype=np.complex128).ravel() for As in tensor_sets for a in As])
    _check(_lib.ttn_set_multiset_state(ctx, len(tensor_sets), flat, offs), ctx)


def ttn_get_multiset_state(ctx, alpha, sizes):
    out = np.zeros(int(sum(sizes)), dtype=np.complex128)
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    _check(_lib.ttn_get_multiset_state(ctx, int(alpha), out, offs), ctx)
    return [out[offs[i]:offs[i + 1]].copy() for i in range(len(sizes))]


def ttn_n_sets(ctx):
    n = C.c_int(0)
    _check(_lib.ttn_n_sets(ctx, C.byref(n)), ctx)
    return n.value


def ttn_set_populations(ctx):
    pops = np.zeros(ttn_n_sets(ctx), dtype=np.float64)
    _check(_lib.ttn_set_populations(ctx, pops), ctx)
    return pops


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, ttn_step_opts):
        return C.byref(opts)
    o = ttn_step_opts(**opts)
    return C.byref(o)


def ttn_step(ctx, dt, nsteps=1, opts=None):
    _check(_lib.ttn_step(ctx, float(dt), int(nsteps), _opts(opts)), ctx)


def ttn_set_coefficients(ctx, coeff):
    coeff = np.ascontiguousarray(coeff, dtype=np.complex128)
    _check(_lib.ttn_set_coefficients(ctx, len(coeff), coeff if coeff.size else np.zeros(1, np.complex128)), ctx)


def ttn_save(ctx) -> bytes:
    n = C.c_size_t(0)
    _check(_lib.ttn_save(ctx, None, C.byref(n)), ctx)
    buf = C.create_string_buffer(n.value)
    _check(_lib.ttn_save(ctx, buf, C.byref(n)), ctx)
    return buf.raw[:n.value]


def ttn_load(ctx, data: bytes):
    buf = C.create_string_buffer(bytes(data), len(data))
    _check(_lib.ttn_load(ctx, buf, len(data)), ctx)


def ttn_ground_state(ctx, nsweeps):
    e = np.zeros(max(1, int(nsweeps)), dtype=np.float64)
    _check(_lib.ttn_ground_state(ctx, int(nsweeps), e), ctx)
    return e[:int(nsweeps)].copy()


def ttn_step_batch(ctxs, dt, nsteps=1, opts=None):
    arr = (_P * len(ctxs))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    st = _lib.ttn_step_batch(arr, len(ctxs), float(dt), int(nsteps), _opts(opts))
    if st != TTN_OK:
        msgs = "; ".join(ttn_last_error(c) for c in ctxs if ttn_last_error(c))
        raise TTNError(st, msgs)


def ttn_reduced_density(ctx, leaf, d):
    out = np.zeros(d * d, dtype=np.complex128)
    _check(_lib.ttn_reduced_density(ctx, int(leaf), out), ctx)
    return out.reshape(d, d)


def ttn_expect(ctx, leaves, ops):
    leaves = np.ascontiguousarray(leaves, dtype=np.int32)
    flat, offs = _flatten(ops)
    out = np.zeros(len(leaves), dtype=np.complex128)
    _check(_lib.ttn_expect(ctx, len(leaves), leaves, flat, offs[:-1].copy(), out), ctx)
    return out


def ttn_norm_energy(ctx):
    n = C.c_double(0.0)
    e = np.zeros(1, dtype=np.complex128)
    _check(_lib.ttn_norm_energy(ctx, C.byref(n), e), ctx)
    return n.value, complex(e[0])


def ttn_vacuum_projection(ctx, keep_leaf, d):
    out = np.zeros(d, dtype=np.complex128)
    _check(_lib.ttn_vacuum_projection(ctx, int(keep_leaf), out), ctx)
    return out


def ttn_get_state(ctx, sizes):
    total = int(np.sum(sizes))
    flat = np.zeros(total, dtype=np.complex128)
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    _check(_lib.ttn_get_state(ctx, flat, offs), ctx)
    return [flat[offs[i]:offs[i + 1]] for i in range(len(sizes))]


def ttn_tree(ctx):
    """(parent, phys_dim, bond_dim) of the context's current tree."""
    n = C.c_int(0)
    _check(_lib.ttn_tree(ctx, C.byref(n), None, None, None), ctx)
    par, phys, bond = (np.zeros(n.value, dtype=np.int32) for _ in range(3))
    _check(_lib.ttn_tree(ctx, C.byref(n), par.ctypes.data, phys.ctypes.data, bond.ctypes.data), ctx)
    return par, phys, bond


def ttn_bond_dims(ctx, n_nodes=None):
    """Bond dimensions (root: 1); the length is the library's node count."""
    return ttn_tree(ctx)[2]


OP_NAMES = {1: "qr_down", 2: "qr_up", 3: "absorb_child", 4: "absorb_parent", 5: "env", 6: "combo",
            7: "evolve", 8: "dot", 9: "trace", 10: "contract_vec", 11: "step_end", 12: "spawn", 13: "eigen", 14: "phase",
            16: "in:heff", 17: "in:gram_schmidt", 18: "in:small_expm", 19: "in:gram", 20: "in:convert"}


def ttn_op_cycles(ctx):
    out = np.zeros(32, dtype=np.uint64)
    _check(_lib.ttn_op_cycles(ctx, out), ctx)
    return {OP_NAMES.get(i, str(i)): int(v) for i, v in enumerate(out) if v}


def ttn_heff_apply(stream, dims, coeff, factor, mat_ptrs, x_ptr, y_ptr):
    """dims: index dimensions; coeff[n_terms]; factor[n_terms, D] (-1 identity);
    mat_ptrs, x_ptr, y_ptr: device addresses (ints)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    coeff = np.ascontiguousarray(coeff, dtype=np.complex128)
    factor = np.ascontiguousarray(factor, dtype=np.int32).reshape(-1)
    mp = (_P * max(1, len(mat_ptrs)))(*[int(a) for a in mat_ptrs])
    _check(_lib.ttn_heff_apply(C.c_void_p(int(stream or 0)), len(dims), dims, len(coeff), coeff, factor,
                               len(mat_ptrs), mp, C.c_void_p(int(x_ptr)), C.c_void_p(int(y_ptr))), None)


def ttn_heff_apply_noalloc(stream, dims, coeff, factor, mat_ptrs, x_ptr, y_ptr):
    """Allocation-free ttn_heff_apply (static device scratch shared by all
    calls; limits and the race between overlapping calls in include/ttn.h)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    coeff = np.ascontiguousarray(coeff, dtype=np.complex128)
    factor = np.ascontiguousarray(factor, dtype=np.int32).reshape(-1)
    mp = (_P * max(1, len(mat_ptrs)))(*[int(a) for a in mat_ptrs])
    _check(_lib.ttn_heff_apply_noalloc(C.c_void_p(int(stream or 0)), len(dims), dims, len(coeff), coeff, factor,
                                       len(mat_ptrs), mp, C.c_void_p(int(x_ptr)), C.c_void_p(int(y_ptr))), None)


def ttn_set_device(device: int):
    _check(_lib.ttn_set_device(int(device)), None)


def ttn_mode_product_c64(stream, L, n, R, M_ptr, x_ptr, y_ptr, w=1.0, accumulate=False, tensor_cores=True):
    """y[l, p, r] (+)= w sum_m M[p, m] x[l, m, r] on device complex64 buffers."""
    w = complex(w)
    _check(_lib.ttn_mode_product_c64(C.c_void_p(int(stream or 0)), int(L), int(n), int(R), C.c_void_p(int(M_ptr)),
                                     C.c_void_p(int(x_ptr)), C.c_void_p(int(y_ptr)), w.real, w.imag,
                                     int(bool(accumulate)), int(bool(tensor_cores))), None)


def ttn_autotune(ctx, dt, steps=2, flags=3):
    ms = C.c_double(0.0)
    _check(_lib.ttn_autotune(ctx, float(dt), int(steps), int(flags), C.byref(ms)), ctx)
    return ms.value


def ttn_tuning(ctx):
    b, n = C.c_int(0), C.c_int(0)
    t, d = C.c_double(0.0), C.c_double(0.0)
    v = np.zeros(65, dtype=np.uint8)
    _check(_lib.ttn_tuning(ctx, C.byref(b), v, C.byref(t), C.byref(d), C.byref(n)), ctx)
    return {"blocks": b.value, "variants": {i: int(x) for i, x in enumerate(v) if x}, "tuned_ms": t.value,
            "default_ms": d.value, "trials": n.value}


def ttn_operator_dims(ctx, n_nodes):
    out = np.zeros(n_nodes, dtype=np.int32)
    _check(_lib.ttn_operator_dims(ctx, out), ctx)
    return out


def ttn_set_tuning(ctx, blocks, variants):
    v = np.zeros(65, dtype=np.uint8)
    for n, x in (variants.items() if isinstance(variants, dict) else enumerate(variants)):
        v[int(n)] = int(x)
    _check(_lib.ttn_set_tuning(ctx, int(blocks), v), ctx)


def ttn_pipe_peaks(stream=0, seconds=0.5):
    """Measured FP32 and FP64 FMA throughput (TFLOP/s) of the current device."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.ttn_pipe_peaks(C.c_void_p(int(stream or 0)), float(seconds), C.byref(a), C.byref(b)), None)
    return a.value, b.value


def ttn_set_cluster(ctx, blocks: int):
    _check(_lib.ttn_set_cluster(ctx, int(blocks)), ctx)


def ttn_get_cluster(ctx) -> int:
    n = C.c_int(0)
    _check(_lib.ttn_get_cluster(ctx, C.byref(n)), ctx)
    return n.value


def ttn_step_stats(ctx, max_stamps=4096):
    steps = C.c_int64(0)
    fl = C.c_double(0.0)
    st = np.zeros(max(1, max_stamps), dtype=np.uint64)
    n = C.c_int(0)
    _check(_lib.ttn_step_stats(ctx, C.byref(steps), C.byref(fl), st, int(max_stamps), C.byref(n)), ctx)
    return steps.value, fl.value, st[:n.value].copy()


def ttn_flop_counts(ctx):
    t, f = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.ttn_flop_counts(ctx, C.byref(t), C.byref(f)), ctx)
    return t.value, f.value


def ttn_set_stream(ctx, stream_handle: int):
    _check(_lib.ttn_set_stream(ctx, C.c_void_p(int(stream_handle))), ctx)


def ttn_device_bytes(ctx):
    n = C.c_size_t(0)
    _check(_lib.ttn_device_bytes(ctx, C.byref(n)), ctx)
    return n.value


def ttn_destroy(ctx):
    _lib.ttn_destroy(ctx)


def _server_check(st, srv):
    if st != TTN_OK:
        m = _lib.ttn_server_last_error(srv)
        raise TTNError(st, m.decode() if m else "")


def ttn_server_create(precision=TTN_MIXED, hbm_budget=0, max_slots=0, slice_ms=0.0, use_graph=1):
    o = ttn_server_opts(int(hbm_budget), int(max_slots), float(slice_ms), int(use_graph))
    h = _P()
    st = _lib.ttn_server_create(int(precision), C.byref(o), C.byref(h))
    if st != TTN_OK:
        raise TTNError(st, "ttn_server_create failed")
    return h


def ttn_server_submit(srv, ctx, dt, nsteps, opts=None):
    t = C.c_int64(0)
    _server_check(_lib.ttn_server_submit(srv, ctx, float(dt), int(nsteps), _opts(opts), C.byref(t)), srv)
    return t.value


def ttn_server_pump(srv):
    r, q = C.c_int(0), C.c_int(0)
    _server_check(_lib.ttn_server_pump(srv, C.byref(r), C.byref(q)), srv)
    return r.value, q.value


def ttn_server_drain(srv):
    _server_check(_lib.ttn_server_drain(srv), srv)


def ttn_server_poll(srv, max_n=4096):
    t = np.zeros(max(1, max_n), dtype=np.int64)
    s = np.zeros(max(1, max_n), dtype=np.int32)
    n = C.c_int(0)
    _server_check(_lib.ttn_server_poll(srv, int(max_n), t, s, C.byref(n)), srv)
    return list(zip(t[:n.value].tolist(), s[:n.value].tolist()))


def ttn_server_get_stats(srv):
    st = ttn_server_stats()
    _server_check(_lib.ttn_server_get_stats(srv, C.byref(st)), srv)
    return {k: getattr(st, k) for k, _ in ttn_server_stats._fields_}


def ttn_server_latencies(srv, max_n=1 << 22):
    out = np.zeros(max(1, max_n), dtype=np.float64)
    n = C.c_int64(0)
    _server_check(_lib.ttn_server_latencies(srv, out, int(max_n), C.byref(n)), srv)
    return out[:n.value].copy()


def ttn_server_last_error(srv) -> str:
    m = _lib.ttn_server_last_error(srv)
    return m.decode() if m else ""


def ttn_server_destroy(srv):
    _lib.ttn_server_destroy(srv)


class Server:
    """Owns one ttn_server (continuous batching of contexts; include/ttn.h)."""

    def __init__(self, precision=TTN_MIXED, hbm_budget=0, max_slots=0, slice_ms=0.0, use_graph=True):
        self.h = ttn_server_create(precision, hbm_budget, max_slots, slice_ms, int(bool(use_graph)))

    def submit(self, ctx, dt, nsteps, opts=None):
        return ttn_server_submit(self.h, ctx.h, dt, nsteps, opts)

    def pump(self):
        return ttn_server_pump(self.h)

    def drain(self):
        ttn_server_drain(self.h)

    def poll(self):
        return ttn_server_poll(self.h)

    def stats(self):
        return ttn_server_get_stats(self.h)

    def latencies(self):
        return ttn_server_latencies(self.h)

    def close(self):
        if self.h:
            ttn_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# convenience wrapper around a context handle
# ---------------------------------------------------------------------------
class TreeView:
    """Tree shape as the library reports it (parent, phys_dim, bond_dim)."""

    def __init__(self, parent, phys_dim, bond_dim):
        self.parent, self.phys_dim, self.bond_dim = parent, phys_dim, bond_dim

    @property
    def n(self):
        return len(self.parent)

    def children(self, z):
        return [c for c in range(z + 1, self.n) if self.parent[c] == z]

    def is_leaf(self, z):
        return self.phys_dim[z] > 0

    def leaves(self):
        return [z for z in range(self.n) if self.phys_dim[z] > 0]


class Context:
    """Owns one ttn_ctx.  ``tree`` is a workloads.Tree (parent/phys_dim/bond_dim)."""

    def __init__(self, tree, precision=TTN_FP64, on_host=False):
        self.tree = tree
        self.precision = precision
        make = ttn_create_host if on_host else ttn_create
        self.h = make(tree.parent, tree.phys_dim, tree.bond_dim, precision)

    def footprint(self):
        return ttn_footprint(self.h)

    def device_bytes(self):
        return ttn_device_bytes(self.h)

    def evict(self):
        ttn_evict(self.h)

    def materialize(self):
        ttn_materialize(self.h)

    def set_state(self, tensors):
        ttn_set_state(self.h, tensors)

    def set_hamiltonian(self, H):
        coeff, term_ptr, leaf, mats, off = H.to_csr()
        ttn_set_sop_hamiltonian(self.h, coeff, term_ptr, leaf, mats, off, H.hermitian)

    def set_multiset_hamiltonian(self, H):
        """H: workloads.MultiSetSOP (terms c_r |bra_r><ket_r| (x) factors)."""
        coeff, term_ptr, leaf, mats, off, bra, ket = H.to_csr()
        ttn_set_multiset_hamiltonian(self.h, H.n_sets, coeff, term_ptr, leaf, mats, off, bra, ket, H.hermitian)

    def set_multiset_state(self, tensor_sets):
        ttn_set_multiset_state(self.h, tensor_sets)

    def n_sets(self):
        return ttn_n_sets(self.h)

    def set_populations(self):
        return ttn_set_populations(self.h)

    def get_multiset_state(self, alpha):
        bond = self.bond_dims()
        dims = [self.mode_dims(z, bond) for z in range(self.tree.n)]
        flat = ttn_get_multiset_state(self.h, alpha, [int(np.prod(d)) for d in dims])
        return [f.reshape(d) for f, d in zip(flat, dims)]

    def step(self, dt, nsteps=1, opts=None):
        ttn_step(self.h, dt, nsteps, opts)

    def autotune(self, dt, steps=2, flags=3):
        """Time candidate launch shapes / contraction routines on this problem
        and keep the fastest; the state is left unchanged."""
        return ttn_autotune(self.h, dt, steps, flags)

    def tuning(self):
        return ttn_tuning(self.h)

    def operator_dims(self):
        """Channels of the hierarchical SOP crossing each bond (index = child)."""
        return ttn_operator_dims(self.h, self.tree.n)

    def set_tuning(self, blocks, variants):
        ttn_set_tuning(self.h, blocks, variants)

    def set_cluster(self, blocks):
        """Thread blocks per instance: 0 = automatic, 1 = one block, 2..16 = a cluster."""
        ttn_set_cluster(self.h, blocks)

    def cluster(self):
        return ttn_get_cluster(self.h)

    def set_coefficients(self, coeff):
        ttn_set_coefficients(self.h, coeff)

    def save(self) -> bytes:
        return ttn_save(self.h)

    def load(self, data: bytes):
        """Replace tree, state and Hamiltonian by a checkpoint's; the tree
        view becomes the checkpoint's tree."""
        ttn_load(self.h, data)
        self.tree = TreeView(*ttn_tree(self.h))

    def ground_state(self, nsweeps=1):
        return ttn_ground_state(self.h, nsweeps)

    def rdm(self, leaf):
        return ttn_reduced_density(self.h, leaf, int(self.tree.phys_dim[leaf]))

    def populations(self, leaves):
        return [np.real(np.diag(self.rdm(l))) for l in leaves]

    def norm_energy(self):
        return ttn_norm_energy(self.h)

    def vacuum_projection(self, keep_leaf):
        return ttn_vacuum_projection(self.h, keep_leaf, int(self.tree.phys_dim[keep_leaf]))

    def bond_dims(self):
        return ttn_bond_dims(self.h, self.tree.n)

    def mode_dims(self, z, bond=None):
        """Index dimensions of node z with the context's current bond dimensions."""
        bond = self.bond_dims() if bond is None else bond
        t = self.tree
        first = [int(t.phys_dim[z])] if t.phys_dim[z] > 0 else [int(bond[c]) for c in t.children(z)]
        return first + [int(bond[z]) if z > 0 else 1]

    def get_state(self):
        bond = self.bond_dims()
        dims = [self.mode_dims(z, bond) for z in range(self.tree.n)]
        flat = ttn_get_state(self.h, [int(np.prod(d)) for d in dims])
        return [f.reshape(d) for f, d in zip(flat, dims)]

    def close(self):
        if self.h:
            ttn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
