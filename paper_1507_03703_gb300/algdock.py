"""Thin ctypes binding of libalgdock (include/algdock.h).

Argument marshalling only: every computation runs in the CUDA library.  Arrays are torch CUDA
tensors (device pointers) or, where the C call accepts host memory, numpy arrays.  The library must
have been built (``paper_1507_03703_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libalgdock.so")

OK, E_INVALID, E_CUDA, E_OOM, E_NUMERIC, E_NOT_CONVERGED, E_STATE = range(7)
CNT_ACCEPTED, CNT_NONFINITE, CNT_OUTSIDE = 0, 1, 2
N_COUNTERS = 4

# Unit conventions of the C ABI: A, kcal/mol, amu, fs, K.
K_RESTRAINT = 10000.0 / 4.184 / 100.0  # 10000 kJ/(mol nm^2) in kcal/(mol A^2)
D0 = 6.0
VMAX_R = 10.0 / 4.184                  # 10 kJ/mol per unit scale factor, in kcal/mol

EXPORTS = [
    "algdock_create", "algdock_destroy", "algdock_set_stream", "algdock_last_error", "algdock_grids_build",
    "algdock_soft_elec_cap", "algdock_grids_load", "algdock_ligand_load", "algdock_states_set",
    "algdock_hmc_cycle", "algdock_energy_force", "algdock_exchange", "algdock_reduced_energies", "algdock_mbar",
    "algdock_mbar_noalloc", "algdock_learned_ntorsions", "algdock_learned_features", "algdock_pose_delta",
    "algdock_mlp_forward", "algdock_mlp_grad", "algdock_mlp_adam", "algdock_propose_learned",
    "algdock_external_moves", "algdock_detect_equilibration", "algdock_state_statistics", "algdock_resample",
    "algdock_mean_pacc", "algdock_receptor_load", "algdock_target_interaction", "algdock_fep",
    "algdock_batch_load", "algdock_batch_layout", "algdock_batch_hmc_cycle", "algdock_batch_tune",
    "algdock_hmc_shape", "algdock_batch_shapes", "algdock_gather_probe", "algdock_grids_load_f64",
    "algdock_energy_force_f64", "algdock_checkpoint_save", "algdock_checkpoint_load", "algdock_mbar_partials",
    "algdock_mbar_update", "algdock_next_temperature", "algdock_next_alpha", "algdock_adapt_dt",
    "algdock_insert_states", "algdock_cycle", "algdock_gemm_bf16", "algdock_params_default", "algdock_set_params",
    "algdock_get_params", "algdock_replicas_init", "algdock_run", "algdock_replicas_get", "algdock_replicas_save",
    "algdock_replicas_load", "algdock_gather_layout",
]

BATCH_CLASSES = 4             # launch classes of a multi-ligand batch
ALPHA_MAX_EXTERNAL = 0.01     # external-coordinate moves only below this alpha ("Sampling")
SIGMA_TRANSLATION = 0.6       # A per dimension ("Sampling")
MLP_NFEAT, MLP_NHID, MLP_NOUT, MLP_DMAX = 64, 256, 360, 22
MLP_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")
MLP_NPARAMS = 64 * 256 + 256 + 256 * 256 + 256 + 256 * 256 + 256 + 256 * 360 + 360
MLP_NWEIGHTS = 64 * 256 + 256 * 256 + 256 * 256 + 256 * 360


def bf16_bits(a):
    """Round float32 values to BF16 (nearest even) and return the 16-bit patterns."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = np.where(finite, u + 0x7FFF + ((u >> 16) & 1), u)
    return ((r >> 16) & 0xFFFF).astype(np.uint16)


def bf16_values(a):
    """The float32 values of the BF16 rounding of a."""
    return (bf16_bits(a).astype(np.uint32) << 16).view(np.float32)


def pack_mlp(params):
    """Flatten a parameter dict (W1 [256][64], b1, ..., W4 [360][256], b4) into the library's FP32
    parameter vector and the BF16 copy of its weight matrices (numpy)."""
    flat = np.concatenate([np.asarray(params[k], dtype=np.float32).ravel() for k in MLP_KEYS])
    w = np.concatenate([np.asarray(params[k], dtype=np.float32).ravel() for k in ("W1", "W2", "W3", "W4")])
    assert flat.size == MLP_NPARAMS and w.size == MLP_NWEIGHTS
    return flat, bf16_bits(w)


def unpack_mlp(flat):
    """Inverse of the FP32 part of pack_mlp."""
    shapes = {"W1": (256, 64), "b1": (256,), "W2": (256, 256), "b2": (256,), "W3": (256, 256), "b3": (256,),
              "W4": (360, 256), "b4": (360,)}
    out, o = {}, 0
    for k in MLP_KEYS:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


class AlgdockError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("algdock status %d: %s" % (status, msg))
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("spacing", C.c_double), ("n", C.c_int32 * 3)]


class LigandC(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("mass", C.c_void_p), ("charge", C.c_void_p), ("rstar", C.c_void_p),
                ("eps", C.c_void_p), ("n_bonds", C.c_int32), ("bonds", C.c_void_p), ("bond_k", C.c_void_p),
                ("bond_r0", C.c_void_p), ("n_angles", C.c_int32), ("angles", C.c_void_p),
                ("angle_k", C.c_void_p), ("angle_theta0", C.c_void_p), ("n_torsions", C.c_int32),
                ("torsions", C.c_void_p), ("torsion_V", C.c_void_p), ("torsion_gamma", C.c_void_p)]


class RestraintC(C.Structure):
    _fields_ = [("site", C.c_double * 3), ("k", C.c_double), ("d0", C.c_double)]


MAX_LEGS = 8


class RunDescC(C.Structure):
    """algdock_run_desc: the legs, chains and per-cycle settings of a run for algdock_cycle."""
    _fields_ = [("n_legs", C.c_int32), ("K", C.c_int32 * MAX_LEGS), ("state_offset", C.c_int32 * MAX_LEGS),
                ("n_chains", C.c_int32), ("n_steps", C.c_int32), ("n_sweeps", C.c_int32), ("max_sep", C.c_int32),
                ("seed", C.c_uint64), ("rep_offset", C.c_int64), ("ladder_offset", C.c_int64),
                ("n_external", C.c_int32), ("alpha_max", C.c_double), ("sigma_ext", C.c_double)]


class ParamsC(C.Structure):
    """algdock_params: the method's adjustable arguments held by a context."""
    _fields_ = [("n_steps", C.c_int32), ("n_sweeps", C.c_int32), ("max_sep", C.c_int32), ("n_external", C.c_int32),
                ("alpha_max", C.c_double), ("sigma_ext", C.c_double), ("mbar_tol", C.c_double),
                ("mbar_max_iter", C.c_int32), ("mbar_precision", C.c_int32), ("checks", C.c_int32)]


class ArrayC(C.Structure):
    """algdock_array: one named array of a checkpoint."""
    _fields_ = [("name", C.c_char * 32), ("dtype", C.c_int32), ("count", C.c_int64), ("data", C.c_void_p)]


# algdock_dtype codes
F32, F64, I32, I64, U8 = 1, 2, 3, 4, 5
_NP_DTYPE = {F32: np.float32, F64: np.float64, I32: np.int32, I64: np.int64, U8: np.uint8}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libalgdock.so and declare its signatures.  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libalgdock.so not built: run paper_1507_03703_gb300.build.build() (needs nvcc)")
    L = C.CDLL(path)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "algdock_create": ([C.c_int, u64, C.POINTER(ParamsC), C.POINTER(vp)], C.c_int),
        "algdock_params_default": ([C.POINTER(ParamsC)], C.c_int),
        "algdock_set_params": ([vp, C.POINTER(ParamsC)], C.c_int),
        "algdock_get_params": ([vp, C.POINTER(ParamsC), C.POINTER(u64)], C.c_int),
        "algdock_replicas_init": ([vp, i32, vp, vp, i32, i64, i64, vp], C.c_int),
        "algdock_run": ([vp, i32, u64, vp], C.c_int),
        "algdock_replicas_get": ([vp, vp, vp, vp, vp, vp], C.c_int),
        "algdock_replicas_save": ([vp, C.c_char_p, u64], C.c_int),
        "algdock_replicas_load": ([vp, C.c_char_p, C.POINTER(u64)], C.c_int),
        "algdock_destroy": ([vp], None),
        "algdock_set_stream": ([vp, vp], C.c_int),
        "algdock_last_error": ([vp], C.c_char_p),
        "algdock_grids_build": ([vp, C.POINTER(GridDesc), i32, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "algdock_soft_elec_cap": ([C.POINTER(LigandC), dbl, C.POINTER(dbl)], C.c_int),
        "algdock_gather_layout": ([C.POINTER(LigandC), vp, vp, vp, vp], C.c_int),
        "algdock_grids_load": ([vp, C.POINTER(GridDesc), vp, vp, vp, dbl, dbl], C.c_int),
        "algdock_ligand_load": ([vp, C.POINTER(LigandC), C.POINTER(RestraintC)], C.c_int),
        "algdock_states_set": ([vp, i32, vp, vp, vp], C.c_int),
        "algdock_hmc_cycle": ([vp, i64, vp, vp, vp, vp, vp, i32, u64, u64, i64, vp], C.c_int),
        "algdock_energy_force": ([vp, i64, vp, vp, vp, vp], C.c_int),
        "algdock_external_moves": ([vp, i64, vp, vp, vp, i32, dbl, dbl, u64, u64, i64, vp, vp], C.c_int),
        "algdock_detect_equilibration": ([vp, i64, i64, vp, i64, i32, vp, vp, vp], C.c_int),
        "algdock_state_statistics": ([vp, i64, vp, i32, vp], C.c_int),
        "algdock_resample": ([vp, i64, vp, i32, i32, i32, u64, C.c_uint32, vp, vp, vp], C.c_int),
        "algdock_mean_pacc": ([vp, i64, vp, vp, i32, i32, vp], C.c_int),
        "algdock_receptor_load": ([vp, i32, vp, vp, vp, vp], C.c_int),
        "algdock_target_interaction": ([vp, i64, vp, vp], C.c_int),
        "algdock_fep": ([vp, i64, vp, i64, vp, i64, dbl, vp], C.c_int),
        "algdock_batch_load": ([vp, i32, vp, vp], C.c_int),
        "algdock_batch_layout": ([vp, i64, vp, i32, i32], C.c_int),
        "algdock_batch_hmc_cycle": ([vp, vp, vp, vp, vp, vp, i32, u64, u64, i64, vp], C.c_int),
        "algdock_batch_tune": ([vp, vp, vp, i32, i32, vp, vp], C.c_int),
        "algdock_hmc_shape": ([vp, vp], C.c_int),
        "algdock_gather_probe": ([vp, i64, i32, u64, vp], C.c_int),
        "algdock_grids_load_f64": ([vp, C.POINTER(GridDesc), vp, vp, vp, dbl, dbl], C.c_int),
        "algdock_energy_force_f64": ([vp, i64, vp, vp, vp, vp], C.c_int),
        "algdock_batch_shapes": ([vp, vp], C.c_int),
        "algdock_exchange": ([vp, i32, i32, i32, vp, vp, vp, i32, i32, u64, u64, i64, vp, vp], C.c_int),
        "algdock_reduced_energies": ([vp, i64, vp, vp, i32, i32, vp], C.c_int),
        "algdock_mbar": ([vp, i32, i64, vp, vp, dbl, i32, i32, vp, C.POINTER(i32)], C.c_int),
        "algdock_mbar_noalloc": ([vp, i32, i64, vp, vp, dbl, i32, i32, vp, C.POINTER(i32)], C.c_int),
        "algdock_learned_ntorsions": ([vp, C.POINTER(i32)], C.c_int),
        "algdock_learned_features": ([vp, i64, vp, vp, vp, vp], C.c_int),
        "algdock_pose_delta": ([vp, i64, vp, vp, vp], C.c_int),
        "algdock_mlp_forward": ([vp, vp, vp, i64, vp, vp], C.c_int),
        "algdock_mlp_grad": ([vp, vp, vp, i64, vp, vp, i32, vp, vp], C.c_int),
        "algdock_mlp_adam": ([vp, vp, vp, vp, vp, vp, i32, C.c_float], C.c_int),
        "algdock_propose_learned": ([vp, vp, vp, i64, vp, vp, vp, i32, i32, u64, u64, i64, vp, vp], C.c_int),
        "algdock_mbar_partials": ([vp, i32, i64, vp, vp, vp, i32, vp], C.c_int),
        "algdock_cycle": ([vp, C.POINTER(RunDescC), u64, vp, vp, vp, vp, vp, vp], C.c_int),
        "algdock_gemm_bf16": ([vp, i32, i32, i32, vp, i32, vp, i32, vp, i32, i32, vp, vp, i32, i32], C.c_int),
        "algdock_mbar_update": ([i32, i32, vp, vp, vp, C.POINTER(dbl)], C.c_int),
        "algdock_next_temperature": ([dbl, dbl, dbl, dbl, C.POINTER(dbl)], C.c_int),
        "algdock_next_alpha": ([dbl, dbl, dbl, dbl, dbl, dbl, dbl, C.POINTER(dbl)], C.c_int),
        "algdock_adapt_dt": ([dbl, dbl, C.POINTER(dbl)], C.c_int),
        "algdock_insert_states": ([i32, vp, vp, vp, vp, vp, dbl, dbl, dbl, i32, C.POINTER(i32), vp, vp, vp, vp],
                                  C.c_int),
        "algdock_checkpoint_save": ([vp, C.c_char_p, u64, u64, i32, C.POINTER(ArrayC)], C.c_int),
        "algdock_checkpoint_load": ([vp, C.c_char_p, C.POINTER(u64), C.POINTER(u64), i32, C.POINTER(ArrayC)],
                                    C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _dev(t, dtype=None, name="array"):
    """Device pointer of a contiguous torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a torch CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    return t.data_ptr()


def _any(a, np_dtype, torch_dtype, name):
    """Pointer to a host numpy array or a device tensor; returns (ptr, keepalive)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                return _dev(a, torch_dtype, name), a
            a = a.numpy()
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np_dtype)
    return arr.ctypes.data, arr


def ligand_struct(lig):
    """Build the C ligand description from any object with the fields of algdock_ligand."""
    keep = []

    def f64(a):
        arr = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(arr)
        return arr.ctypes.data

    def i32(a, w):
        arr = np.ascontiguousarray(np.asarray(a).reshape(-1, w), dtype=np.int32)
        keep.append(arr)
        return arr.ctypes.data

    s = LigandC()
    s.n_atoms = int(len(lig.mass))
    s.mass, s.charge, s.rstar, s.eps = f64(lig.mass), f64(lig.charge), f64(lig.rstar), f64(lig.eps)
    s.n_bonds = int(np.asarray(lig.bonds).reshape(-1, 2).shape[0])
    s.bonds, s.bond_k, s.bond_r0 = i32(lig.bonds, 2), f64(lig.bond_k), f64(lig.bond_r0)
    s.n_angles = int(np.asarray(lig.angles).reshape(-1, 3).shape[0])
    s.angles, s.angle_k, s.angle_theta0 = i32(lig.angles, 3), f64(lig.angle_k), f64(lig.angle_theta0)
    s.n_torsions = int(np.asarray(lig.torsions).reshape(-1, 4).shape[0])
    s.torsions, s.torsion_V, s.torsion_gamma = i32(lig.torsions, 4), f64(lig.torsion_V), f64(lig.torsion_gamma)
    return s, keep


def soft_elec_cap(lig, vmax_r: float = VMAX_R) -> float:
    L = load_library()
    s, keep = ligand_struct(lig)
    out = C.c_double()
    st = L.algdock_soft_elec_cap(C.byref(s), float(vmax_r), C.byref(out))
    if st != OK:
        raise AlgdockError(st, "soft_elec_cap: invalid ligand")
    return out.value


def gather_layout(lig):
    """algdock_gather_layout: the bonded-force layout of lig's topology, as a dict of term_order
    [n_terms], slots [n_slots], lane_run [32] and wavefronts (input order, layout)."""
    L = load_library()
    s, keep = ligand_struct(lig)
    n_terms = s.n_bonds + s.n_angles + s.n_torsions
    n_slots = 2 * s.n_bonds + 3 * s.n_angles + 4 * s.n_torsions
    order = np.zeros(max(n_terms, 1), np.int32)
    slots = np.zeros(max(n_slots, 1), np.uint16)
    lane_run = np.zeros(32, np.int32)
    wf = np.zeros(2, np.int32)
    st = L.algdock_gather_layout(C.byref(s), order.ctypes.data, slots.ctypes.data, lane_run.ctypes.data,
                                 wf.ctypes.data)
    if st != OK:
        raise AlgdockError(st, "gather_layout: invalid topology")
    return {"term_order": order[:n_terms], "slots": slots[:n_slots], "lane_run": lane_run,
            "wavefronts": (int(wf[0]), int(wf[1]))}


def grid_desc(grid) -> GridDesc:
    d = GridDesc()
    for k in range(3):
        d.origin[k] = float(grid.origin[k])
        d.n[k] = int(grid.n[k])
    d.spacing = float(grid.spacing)
    return d


def mbar_update(pairs, f_old):
    """algdock_mbar_update: pairs [n_parts][K][2] (numpy, merged in that order), f_old [K] ->
    (f_new [K], max |f_new - f_old|)."""
    L = load_library()
    pairs = np.ascontiguousarray(pairs, dtype=np.float64)
    f_old = np.ascontiguousarray(f_old, dtype=np.float64)
    n_parts, K = pairs.shape[0], pairs.shape[1]
    f_new = np.empty(K)
    d = C.c_double()
    st = L.algdock_mbar_update(K, n_parts, pairs.ctypes.data, f_old.ctypes.data, f_new.ctypes.data, C.byref(d))
    if st != OK:
        raise AlgdockError(st, "mbar_update: bad arguments")
    return f_new, d.value


def _array_c(name, a):
    """algdock_array for a contiguous torch tensor (device or host) or numpy array."""
    code = None
    if hasattr(a, "data_ptr"):
        import torch
        tmap = {torch.float32: F32, torch.float64: F64, torch.int32: I32, torch.int64: I64, torch.uint8: U8}
        if not a.is_contiguous():
            raise ValueError("checkpoint array %s must be contiguous" % name)
        code, ptr, n = tmap.get(a.dtype), a.data_ptr(), a.numel()
    else:
        if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
            raise ValueError("checkpoint array %s must be a C-contiguous numpy array" % name)
        code = {np.dtype(v): k for k, v in _NP_DTYPE.items()}.get(a.dtype)
        ptr, n = a.ctypes.data, a.size
    if code is None:
        raise ValueError("checkpoint array %s has an unsupported dtype" % name)
    r = ArrayC()
    r.name = name.encode()
    r.dtype, r.count, r.data = code, int(n), ptr if n else None
    return r


def _ck_check(ctx, st, what):
    if st != OK:
        msg = ctx.last_error() if ctx is not None else what + " failed"
        raise AlgdockError(st, msg)


def checkpoint_save(ctx, path, seed, cycle, arrays):
    """algdock_checkpoint_save: arrays is a dict name -> tensor / ndarray (ctx may be None)."""
    L = load_library()
    items = list(arrays.items())
    arr = (ArrayC * max(1, len(items)))(*[_array_c(k, v) for k, v in items])
    _ck_check(ctx, L.algdock_checkpoint_save(ctx.h if ctx is not None else None, str(path).encode(), int(seed),
                                             int(cycle), len(items), arr), "checkpoint_save")


def checkpoint_query(ctx, path, names):
    """dtype code and element count of each named array of a checkpoint (count -1 if absent)."""
    L = load_library()
    arr = (ArrayC * max(1, len(names)))()
    for i, n in enumerate(names):
        arr[i].name = n.encode()
        arr[i].data = None
    _ck_check(ctx, L.algdock_checkpoint_load(ctx.h if ctx is not None else None, str(path).encode(), None, None,
                                             len(names), arr), "checkpoint_query")
    return {n: (arr[i].dtype, arr[i].count) for i, n in enumerate(names)}


def checkpoint_load(ctx, path, arrays):
    """algdock_checkpoint_load into the given buffers (dict name -> tensor / ndarray); returns
    (seed, cycle).  With a context, its state table is restored too."""
    L = load_library()
    items = list(arrays.items())
    arr = (ArrayC * max(1, len(items)))(*[_array_c(k, v) for k, v in items])
    seed, cycle = C.c_uint64(), C.c_uint64()
    _ck_check(ctx, L.algdock_checkpoint_load(ctx.h if ctx is not None else None, str(path).encode(), C.byref(seed),
                                             C.byref(cycle), len(items), arr), "checkpoint_load")
    return seed.value, cycle.value


def default_params(**fields) -> ParamsC:
    """algdock_params_default, with the given fields replaced."""
    p = ParamsC()
    load_library().algdock_params_default(C.byref(p))
    for k, v in fields.items():
        if k not in dict(ParamsC._fields_):
            raise TypeError("unknown algdock_params field %r" % k)
        setattr(p, k, v)
    return p


def _ptr(a, td, name):
    """Data pointer of a contiguous torch tensor (device or host) or C-contiguous numpy array."""
    import torch
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if a.dtype != td or not a.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor" % (name, td))
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype == np.dtype(str(td)[6:])):
        raise ValueError("%s must be a C-contiguous %s array" % (name, td))
    return a.ctypes.data


class Context:
    """One algdock_ctx on a CUDA device.  Method names follow the C calls without the prefix."""

    def __init__(self, device: int = 0, seed: int = 0, **params):
        """params: any field of algdock_params (n_steps, n_sweeps, max_sep, n_external, alpha_max,
        sigma_ext, mbar_tol, mbar_max_iter, mbar_precision, checks); the rest keep their defaults."""
        self._L = load_library()
        h = C.c_void_p()
        p = default_params(**params)
        st = self._L.algdock_create(int(device), int(seed), C.byref(p), C.byref(h))
        if st != OK:
            raise AlgdockError(st, "algdock_create(%d) failed" % device)
        self.h = h
        self.device = device
        self.n_atoms = None
        self.K = 0

    def close(self):
        if getattr(self, "h", None):
            self._L.algdock_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise AlgdockError(st, self._L.algdock_last_error(self.h).decode())
        return st

    def last_error(self) -> str:
        return self._L.algdock_last_error(self.h).decode()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream (or None for the legacy default stream)."""
        ptr = None if stream is None else C.c_void_p(stream.cuda_stream)
        self._check(self._L.algdock_set_stream(self.h, ptr))
        self.stream = stream

    # ---------------------------------------------------------------- grids
    def grids_build(self, grid, receptor, ljr, lja, elec):
        """Direct-sum raw grids into device float tensors [nz, ny, nx]."""
        d = grid_desc(grid)
        px, kx = _any(receptor.xyz, np.float64, None, "xyz")
        pr, kr = _any(receptor.rstar, np.float64, None, "rstar")
        pe, ke = _any(receptor.eps, np.float64, None, "eps")
        pq, kq = _any(receptor.charge, np.float64, None, "q")
        import torch
        n = int(np.asarray(receptor.rstar).shape[0])
        self._check(self._L.algdock_grids_build(self.h, C.byref(d), n, px, pr, pe, pq,
                                                _dev(ljr, torch.float32, "ljr"), _dev(lja, torch.float32, "lja"),
                                                _dev(elec, torch.float32, "elec")))

    def grids_load(self, grid, ljr, lja, elec, vmax_r=VMAX_R, vmax_e=None, ligand=None):
        """Raw grids (numpy float32 host arrays or CUDA float32 tensors).  vmax_e defaults to the
        soft electrostatic cap of `ligand`."""
        import torch
        if vmax_e is None:
            vmax_e = soft_elec_cap(ligand, vmax_r) if ligand is not None else math.inf
        d = grid_desc(grid)
        p1, k1 = _any(ljr, np.float32, torch.float32, "ljr")
        p2, k2 = _any(lja, np.float32, torch.float32, "lja")
        p3, k3 = _any(elec, np.float32, torch.float32, "elec")
        self._check(self._L.algdock_grids_load(self.h, C.byref(d), p1, p2, p3, float(vmax_r), float(vmax_e)))

    def grids_load_f64(self, grid, ljr, lja, elec, vmax_r=VMAX_R, vmax_e=None, ligand=None):
        """FP64 lattices for the all-FP64 path from raw FP64 grids (numpy or CUDA float64)."""
        import torch
        if vmax_e is None:
            vmax_e = soft_elec_cap(ligand, vmax_r) if ligand is not None else math.inf
        d = grid_desc(grid)
        p1, k1 = _any(ljr, np.float64, torch.float64, "ljr")
        p2, k2 = _any(lja, np.float64, torch.float64, "lja")
        p3, k3 = _any(elec, np.float64, torch.float64, "elec")
        self._check(self._L.algdock_grids_load_f64(self.h, C.byref(d), p1, p2, p3, float(vmax_r), float(vmax_e)))

    def energy_force_f64(self, x, state_of=None, force=None, comps=None):
        """All-FP64 components [N, 4] (and forces [N, n_atoms, 3] if a force tensor is given)."""
        import torch
        N = int(x.shape[0])
        if comps is None:
            comps = torch.empty((N, 4), dtype=torch.float64, device=x.device)
        self._check(self._L.algdock_energy_force_f64(self.h, N, _dev(state_of, torch.int32, "state_of"),
                                                     _dev(x, torch.float32, "x"), _dev(force, torch.float64, "force"),
                                                     _dev(comps, torch.float64, "comps")))
        return comps

    def gather_probe(self, n_cells, soft=True, seed=1, sink=None):
        """Enqueue n_cells random 8-corner lattice gathers (the gather roofline's peak probe)."""
        import torch
        if sink is None:
            sink = torch.zeros(1, dtype=torch.float32, device="cuda:%d" % self.device)
        self._check(self._L.algdock_gather_probe(self.h, int(n_cells), 1 if soft else 0, int(seed),
                                                 _dev(sink, torch.float32, "sink")))
        return sink

    # ---------------------------------------------------------------- ligand and states
    def ligand_load(self, lig, site, k=K_RESTRAINT, d0=D0):
        s, keep = ligand_struct(lig)
        r = RestraintC()
        for i in range(3):
            r.site[i] = float(site[i])
        r.k, r.d0 = float(k), float(d0)
        self._check(self._L.algdock_ligand_load(self.h, C.byref(s), C.byref(r)))
        self.n_atoms = s.n_atoms

    def states_set(self, T, alpha, dt_fs):
        T = np.ascontiguousarray(T, dtype=np.float64)
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        dt = np.ascontiguousarray(dt_fs, dtype=np.float64)
        if not (T.shape == a.shape == dt.shape) or T.ndim != 1:
            raise ValueError("T, alpha, dt must be 1-D of equal length")
        self._check(self._L.algdock_states_set(self.h, T.size, T.ctypes.data, a.ctypes.data, dt.ctypes.data))
        self.K = int(T.size)

    # ---------------------------------------------------------------- sampling
    def hmc_cycle(self, state_of, x, comps, dH=None, accepted=None, n_steps=50, seed=0, cycle=0, rep_offset=0,
                  counters=None):
        import torch
        n_rep = int(state_of.numel())
        self._check(self._L.algdock_hmc_cycle(
            self.h, n_rep, _dev(state_of, torch.int32, "state_of"), _dev(x, torch.float32, "x"),
            _dev(comps, torch.float64, "comps"), _dev(dH, torch.float64, "dH"),
            _dev(accepted, torch.uint8, "accepted"), int(n_steps), int(seed), int(cycle), int(rep_offset),
            _dev(counters, torch.int64, "counters")))

    # ---------------------------------------------------------------- multi-ligand batches
    def batch_load(self, ligands, site, k=K_RESTRAINT, d0=D0):
        """Load many ligands (one restraint) for batched HMC."""
        structs, keep = [], []
        for lig in ligands:
            st, kp = ligand_struct(lig)
            structs.append(st)
            keep.append(kp)
        arr = (LigandC * len(structs))(*structs)
        r = RestraintC()
        for i in range(3):
            r.site[i] = float(site[i])
        r.k, r.d0 = float(k), float(d0)
        self._check(self._L.algdock_batch_load(self.h, len(structs), arr, C.byref(r)))
        self.batch_atoms = [int(st.n_atoms) for st in structs]

    def batch_layout(self, lig_of, x_stride, uniform=False):
        """Replica r runs ligand lig_of[r]; positions are stored x_stride atoms apart."""
        lo = np.ascontiguousarray(lig_of, dtype=np.int32)
        self._check(self._L.algdock_batch_layout(self.h, int(lo.size), lo.ctypes.data, int(x_stride),
                                                 1 if uniform else 0))
        self.batch_n_rep = int(lo.size)

    def batch_hmc_cycle(self, state_of, x, comps, dH=None, accepted=None, n_steps=50, seed=0, cycle=0, rep_offset=0,
                        counters=None):
        import torch
        self._check(self._L.algdock_batch_hmc_cycle(
            self.h, _dev(state_of, torch.int32, "state_of"), _dev(x, torch.float32, "x"),
            _dev(comps, torch.float64, "comps"), _dev(dH, torch.float64, "dH"),
            _dev(accepted, torch.uint8, "accepted"), int(n_steps), int(seed), int(cycle), int(rep_offset),
            _dev(counters, torch.int64, "counters")))

    def hmc_shape(self):
        """(replicas per block, pair table staged) of the one-ligand HMC kernel."""
        out = (C.c_int32 * 2)()
        self._check(self._L.algdock_hmc_shape(self.h, out))
        return out[0], bool(out[1])

    def batch_shapes(self):
        """[(replicas per block, pair table staged)] per batch class ((0, False) if empty)."""
        out = (C.c_int32 * (2 * BATCH_CLASSES))()
        self._check(self._L.algdock_batch_shapes(self.h, out))
        return [(out[2 * k], bool(out[2 * k + 1])) for k in range(BATCH_CLASSES)]

    def batch_tune(self, state_of, x, n_steps=50, n_timed=3):
        """Choose each class's launch shape by timing the whole batch launch.  Returns
        ([(replicas per block, table staged)] per class, ms per launch of the chosen shapes);
        classes: <= 32 atoms, 33-64 with the pair table fitting 16-replica blocks, other 33-64,
        65-96."""
        import torch
        chosen = (C.c_int32 * (2 * BATCH_CLASSES))()
        ms = C.c_float()
        self._check(self._L.algdock_batch_tune(self.h, _dev(state_of, torch.int32, "state_of"),
                                               _dev(x, torch.float32, "x"), int(n_steps), int(n_timed), chosen,
                                               C.byref(ms)))
        return [(chosen[2 * k], bool(chosen[2 * k + 1])) for k in range(BATCH_CLASSES)], ms.value

    def external_moves(self, state_of, x, comps, n_moves=20, seed=0, cycle=0, alpha_max=ALPHA_MAX_EXTERNAL,
                       sigma=SIGMA_TRANSLATION, rep_offset=0, accepted=None, counters=None):
        """External-coordinate moves (random rotation about the COM + Gaussian translation,
        Metropolis) for the replicas whose state has alpha < alpha_max; x and comps in place."""
        import torch
        self._check(self._L.algdock_external_moves(
            self.h, int(state_of.numel()), _dev(state_of, torch.int32, "state_of"), _dev(x, torch.float32, "x"),
            _dev(comps, torch.float64, "comps"), int(n_moves), float(alpha_max), float(sigma), int(seed), int(cycle),
            int(rep_offset), _dev(accepted, torch.int32, "accepted"), _dev(counters, torch.int64, "counters")))

    def detect_equilibration(self, series, stride=1, n_cand=None, g=None, t0_best=None, neff_best=None):
        """series [T][S] float64 (device): per series the statistical inefficiency of each candidate
        tail (g [S][n_cand]), the start maximising N/g (t0_best [S] int64) and that N/g.  Returns
        (g, t0_best, neff_best) as device tensors."""
        import torch
        T, S = int(series.shape[0]), int(series.numel() // max(1, series.shape[0]))
        if n_cand is None:
            n_cand = (T - 2) // int(stride) + 1
        dev = series.device
        g = torch.empty((S, n_cand), dtype=torch.float64, device=dev) if g is None else g
        t0_best = torch.empty(S, dtype=torch.int64, device=dev) if t0_best is None else t0_best
        neff_best = torch.empty(S, dtype=torch.float64, device=dev) if neff_best is None else neff_best
        self._check(self._L.algdock_detect_equilibration(
            self.h, T, S, _dev(series, torch.float64, "series"), int(stride), int(n_cand),
            _dev(g, torch.float64, "g"), _dev(t0_best, torch.int64, "t0_best"),
            _dev(neff_best, torch.float64, "neff_best")))
        return g, t0_best, neff_best

    def state_statistics(self, comps, k):
        """{sigma[U_L + U_I], sigma[Psi_sg], sigma[Psi_g], sigma[u_k]} (numpy) over comps [N][4]."""
        import torch
        out = np.zeros(4)
        self._check(self._L.algdock_state_statistics(self.h, int(comps.shape[0]), _dev(comps, torch.float64, "comps"),
                                                     int(k), out.ctypes.data))
        return out

    def resample(self, comps, k_from, k_to, n_out, seed, counter, x_in=None, x_out=None, idx=None):
        import torch
        self._check(self._L.algdock_resample(
            self.h, int(comps.shape[0]), _dev(comps, torch.float64, "comps"), int(k_from), int(k_to), int(n_out),
            int(seed), int(counter) & 0xFFFFFFFF, _dev(x_in, torch.float32, "x_in"), _dev(x_out, torch.float32, "x_out"),
            _dev(idx, torch.int64, "idx")))

    def mean_pacc(self, comps_a, comps_b, ka, kb):
        import torch
        p = C.c_double()
        self._check(self._L.algdock_mean_pacc(self.h, int(comps_a.shape[0]), _dev(comps_a, torch.float64, "comps_a"),
                                              _dev(comps_b, torch.float64, "comps_b"), int(ka), int(kb), C.byref(p)))
        return p.value

    def receptor_load(self, receptor):
        """Receptor atoms of the target force field (host numpy or CUDA float64 arrays)."""
        px, kx = _any(receptor.xyz, np.float64, None, "xyz")
        pr, kr = _any(receptor.rstar, np.float64, None, "rstar")
        pe, ke = _any(receptor.eps, np.float64, None, "eps")
        pq, kq = _any(receptor.charge, np.float64, None, "q")
        n = int(len(receptor.rstar))
        self._check(self._L.algdock_receptor_load(self.h, n, px, pr, pe, pq))

    def target_interaction(self, x, psi=None):
        """Target-force-field receptor-ligand energy psi_T [N] (float64, kcal/mol) of the
        configurations x [N, n_atoms, 3] (CUDA float32)."""
        import torch
        N = int(x.shape[0])
        if psi is None:
            psi = torch.empty(N, dtype=torch.float64, device=x.device)
        self._check(self._L.algdock_target_interaction(self.h, N, _dev(x, torch.float32, "x"),
                                                       _dev(psi, torch.float64, "psi")))
        return psi

    def fep(self, u_target, u_sampling=None, beta=1.0):
        """Zwanzig estimate f = -ln <exp(-beta (u_target - u_sampling))> over the samples (1-D CUDA
        float64 tensors, any stride, e.g. a column of the components).  Returns a dict with f, its
        standard error for independent samples, the Kish n_eff and the smallest reduced difference."""
        import torch

        def strided(t, name):
            if t is None:
                return None, 0
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 1:
                raise TypeError("%s must be a 1-D CUDA float64 tensor" % name)
            return t.data_ptr(), int(t.stride(0))

        pt, st = strided(u_target, "u_target")
        ps, ss = strided(u_sampling, "u_sampling")
        if u_sampling is not None and u_sampling.shape[0] != u_target.shape[0]:
            raise ValueError("u_target and u_sampling differ in length")
        out = (C.c_double * 4)()
        self._check(self._L.algdock_fep(self.h, int(u_target.shape[0]), pt, st, ps, ss, float(beta), out))
        return {"f": out[0], "sigma": out[1], "n_eff": out[2], "du_min": out[3]}

    def energy_force(self, state_of, x, force, comps=None):
        import torch
        self._check(self._L.algdock_energy_force(
            self.h, int(state_of.numel()), _dev(state_of, torch.int32, "state_of"), _dev(x, torch.float32, "x"),
            _dev(force, torch.float32, "force"), _dev(comps, torch.float64, "comps")))

    def exchange(self, K, state_offset, comps, config_of, state_of=None, n_sweeps=25, max_sep=5, seed=0, cycle=0,
                 ladder_offset=0, attempts=None, accepts=None):
        import torch
        n_ladders = int(config_of.numel()) // int(K)
        self._check(self._L.algdock_exchange(
            self.h, n_ladders, int(K), int(state_offset), _dev(comps, torch.float64, "comps"),
            _dev(config_of, torch.int32, "config_of"), _dev(state_of, torch.int32, "state_of"), int(n_sweeps),
            int(max_sep), int(seed), int(cycle), int(ladder_offset), _dev(attempts, torch.int64, "attempts"),
            _dev(accepts, torch.int64, "accepts")))

    # ---------------------------------------------------------------- estimation
    def reduced_energies(self, N, x=None, comps=None, k_begin=0, k_count=0, u_kn=None):
        import torch
        self._check(self._L.algdock_reduced_energies(
            self.h, int(N), _dev(x, torch.float32, "x"), _dev(comps, torch.float64, "comps"), int(k_begin),
            int(k_count), _dev(u_kn, torch.float64, "u_kn")))

    def mbar(self, u_kn, N_k, tol=1e-10, max_iter=10000, precision_mode=0, raise_on_nonconvergence=True):
        """Returns (f_k numpy [K], iterations)."""
        import torch
        K, N = int(u_kn.shape[0]), int(u_kn.shape[1])
        Nk = np.ascontiguousarray(N_k, dtype=np.int64)
        f = np.zeros(K)
        it = C.c_int32()
        st = self._L.algdock_mbar(self.h, K, N, _dev(u_kn, torch.float64, "u_kn"), Nk.ctypes.data, float(tol),
                                  int(max_iter), int(precision_mode), f.ctypes.data, C.byref(it))
        if st == E_NOT_CONVERGED and not raise_on_nonconvergence:
            return f, -1
        self._check(st)
        return f, it.value

    # ---------------------------------------------------------------- learned proposal
    def cycle(self, legs, n_chains, cycle, x, comps, state_of, config_of, n_steps=50, n_sweeps=25, max_sep=5,
              seed=0, rep_offset=0, ladder_offset=0, counters=None, u_kn=None, n_external=0,
              alpha_max=ALPHA_MAX_EXTERNAL, sigma=SIGMA_TRANSLATION):
        """algdock_cycle: one HMC trial of every replica, the external-coordinate moves (n_external > 0),
        then the exchange sweeps of every ladder (and the snapshot's u_kn if given).  legs: [(K,
        state_offset), ...].  Each array is a device tensor or host memory (a CPU tensor, ideally
        pinned, or a numpy array), updated in place."""
        import torch
        d = RunDescC()
        d.n_legs = len(legs)
        for i, (K, off) in enumerate(legs):
            d.K[i], d.state_offset[i] = int(K), int(off)
        d.n_chains, d.n_steps, d.n_sweeps, d.max_sep = int(n_chains), int(n_steps), int(n_sweeps), int(max_sep)
        d.seed, d.rep_offset, d.ladder_offset = int(seed), int(rep_offset), int(ladder_offset)
        d.n_external, d.alpha_max, d.sigma_ext = int(n_external), float(alpha_max), float(sigma)
        self._check(self._L.algdock_cycle(
            self.h, C.byref(d), int(cycle), _ptr(x, torch.float32, "x"), _ptr(comps, torch.float64, "comps"),
            _ptr(state_of, torch.int32, "state_of"), _ptr(config_of, torch.int32, "config_of"),
            _ptr(counters, torch.int64, "counters"), _ptr(u_kn, torch.float64, "u_kn")))

    # ------------------------------------------------------------ the context's own run
    def params(self) -> dict:
        """The context's algdock_params as a dict, and its seed under "seed"."""
        p, seed = ParamsC(), C.c_uint64()
        self._check(self._L.algdock_get_params(self.h, C.byref(p), C.byref(seed)))
        out = {name: getattr(p, name) for name, _ in ParamsC._fields_}
        out["seed"] = seed.value
        return out

    def set_params(self, **fields):
        """algdock_set_params with the given fields replaced in the context's current params."""
        p = ParamsC()
        self._check(self._L.algdock_get_params(self.h, C.byref(p), None))
        for k, v in fields.items():
            if k not in dict(ParamsC._fields_):
                raise TypeError("unknown algdock_params field %r" % k)
            setattr(p, k, v)
        self._check(self._L.algdock_set_params(self.h, C.byref(p)))

    def replicas_init(self, legs, n_chains, x0, rep_offset=0, ladder_offset=0):
        """algdock_replicas_init: legs [(K, state_offset), ...]; x0 [R][n_atoms][3] float32, a device or
        host tensor or numpy array, R = n_chains * sum(K)."""
        import torch
        K = (C.c_int32 * len(legs))(*[int(k) for k, _ in legs])
        off = (C.c_int32 * len(legs))(*[int(o) for _, o in legs])
        self._replica_legs = [(int(k), int(o)) for k, o in legs]
        self._replica_chains = int(n_chains)
        self._check(self._L.algdock_replicas_init(self.h, len(legs), K, off, int(n_chains), int(rep_offset),
                                                  int(ladder_offset), _ptr(x0, torch.float32, "x0")))

    def ukn_words(self) -> int:
        """Doubles of one cycle's snapshot for the context's replicas (sum over legs of K^2 n_chains)."""
        return sum(K * K * self._replica_chains for K, _ in self._replica_legs)

    def run(self, n_cycles, first_cycle=0, u_kn=None):
        """algdock_run: n_cycles cycles over the context's replicas; u_kn (may be None) a float64
        device or host array of n_cycles * ukn_words() doubles."""
        import torch
        self._check(self._L.algdock_run(self.h, int(n_cycles), int(first_cycle), _ptr(u_kn, torch.float64, "u_kn")))

    def replicas_get(self, x=None, comps=None, state_of=None, config_of=None, counters=None):
        """algdock_replicas_get into the given arrays (device or host; None skips)."""
        import torch
        self._check(self._L.algdock_replicas_get(
            self.h, _ptr(x, torch.float32, "x"), _ptr(comps, torch.float64, "comps"),
            _ptr(state_of, torch.int32, "state_of"), _ptr(config_of, torch.int32, "config_of"),
            _ptr(counters, torch.int64, "counters")))

    def replicas_save(self, path, next_cycle):
        self._check(self._L.algdock_replicas_save(self.h, str(path).encode(), int(next_cycle)))

    def replicas_load(self, path) -> int:
        """algdock_replicas_load; returns the stored next cycle."""
        nxt = C.c_uint64()
        self._check(self._L.algdock_replicas_load(self.h, str(path).encode(), C.byref(nxt)))
        # the layout the context restored: n_legs, n_chains, rep_offset, ladder_offset, K[], offsets[]
        _, count = checkpoint_query(None, path, ["replicas.layout"])["replicas.layout"]
        w = np.zeros(count, dtype=np.int64)
        checkpoint_load(None, path, {"replicas.layout": w})
        n_legs = int(w[0])
        self._replica_chains = int(w[1])
        self._replica_legs = [(int(w[4 + l]), int(w[4 + n_legs + l])) for l in range(n_legs)]
        return nxt.value

    def gemm_bf16(self, A, B, C, epilogue=0, bias=None, mask=None, n_split=1):
        """algdock_gemm_bf16: C = epi(A . B^T) on tcgen05; A [M][K], B [N][K] bfloat16 (or int16 bit
        patterns) device tensors, C [M][N] (or [slices][M][N] with n_split) float32 / bfloat16."""
        import torch
        M, K = A.shape
        N = B.shape[0]
        self._check(self._L.algdock_gemm_bf16(
            self.h, int(M), int(N), int(K), A.data_ptr(), int(A.stride(0)), B.data_ptr(), int(B.stride(0)),
            C.data_ptr(), int(N), int(epilogue), bias.data_ptr() if bias is not None else None,
            mask.data_ptr() if mask is not None else None, int(N), int(n_split)))

    def mbar_partials(self, u_kn, N_k, f, precision_mode=0):
        """This process's (max, sum) pair per state of one MBAR iteration ([K][2] numpy)."""
        import torch
        K = len(N_k)
        N = int(u_kn.shape[1]) if u_kn is not None and u_kn.numel() else 0
        Nk = np.ascontiguousarray(N_k, dtype=np.int64)
        fa = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty((K, 2))
        self._check(self._L.algdock_mbar_partials(self.h, K, N, _dev(u_kn, torch.float64, "u_kn") if N else None,
                                                  Nk.ctypes.data, fa.ctypes.data, int(precision_mode),
                                                  out.ctypes.data))
        return out

    def learned_ntorsions(self):
        T = C.c_int32()
        self._check(self._L.algdock_learned_ntorsions(self.h, C.byref(T)))
        return T.value

    def learned_features(self, state_of, x, comps, feat):
        import torch
        self._check(self._L.algdock_learned_features(
            self.h, int(state_of.numel()), _dev(state_of, torch.int32, "state_of"), _dev(x, torch.float32, "x"),
            _dev(comps, torch.float64, "comps"), _dev(feat, torch.float32, "feat")))

    def pose_delta(self, x, y, delta):
        import torch
        self._check(self._L.algdock_pose_delta(self.h, int(x.shape[0]), _dev(x, torch.float32, "x"),
                                               _dev(y, torch.float32, "y"), _dev(delta, torch.float32, "delta")))

    def mlp_forward(self, params, wbf16, feat, out):
        import torch
        self._check(self._L.algdock_mlp_forward(self.h, _dev(params, torch.float32, "params"),
                                                _dev(wbf16, torch.int16, "wbf16"), int(feat.shape[0]),
                                                _dev(feat, torch.float32, "feat"), _dev(out, torch.float32, "out")))

    def mlp_grad(self, params, wbf16, feat, delta, D, grad, loss=None):
        import torch
        self._check(self._L.algdock_mlp_grad(self.h, _dev(params, torch.float32, "params"),
                                             _dev(wbf16, torch.int16, "wbf16"), int(feat.shape[0]),
                                             _dev(feat, torch.float32, "feat"), _dev(delta, torch.float32, "delta"),
                                             int(D), _dev(grad, torch.float32, "grad"),
                                             _dev(loss, torch.float32, "loss")))

    def mlp_adam(self, params, wbf16, grad, m, v, step, lr):
        import torch
        self._check(self._L.algdock_mlp_adam(self.h, _dev(params, torch.float32, "params"),
                                             _dev(wbf16, torch.int16, "wbf16"), _dev(grad, torch.float32, "grad"),
                                             _dev(m, torch.float32, "m"), _dev(v, torch.float32, "v"), int(step),
                                             float(lr)))

    def propose_learned(self, params, wbf16, state_of, x, comps, n_moves, seed=0, cycle=0, rep_offset=0,
                        accepted=None, counters=None, n_torsions=-1):
        import torch
        self._check(self._L.algdock_propose_learned(
            self.h, _dev(params, torch.float32, "params"), _dev(wbf16, torch.int16, "wbf16"), int(state_of.numel()),
            _dev(state_of, torch.int32, "state_of"), _dev(x, torch.float32, "x"), _dev(comps, torch.float64, "comps"),
            int(n_moves), int(n_torsions), int(seed), int(cycle), int(rep_offset), _dev(accepted, torch.int32, "accepted"),
            _dev(counters, torch.int64, "counters")))

    def mbar_noalloc(self, u_kn, N_k, tol=1e-10, max_iter=10000, precision_mode=0):
        """algdock_mbar_noalloc: MBAR whose scratch is the library's fixed device array (for callers
        that cannot allocate device memory).  Returns (f_k numpy [K], iterations)."""
        import torch
        K, N = int(u_kn.shape[0]), int(u_kn.shape[1])
        Nk = np.ascontiguousarray(N_k, dtype=np.int64)
        f = np.zeros(K)
        it = C.c_int32()
        self._check(self._L.algdock_mbar_noalloc(self.h, K, N, _dev(u_kn, torch.float64, "u_kn"), Nk.ctypes.data,
                                                 float(tol), int(max_iter), int(precision_mode), f.ctypes.data,
                                                 C.byref(it)))
        return f, it.value
