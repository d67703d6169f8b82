"""FP64 CPU oracle (test infrastructure).

A ctypes binding over ``oracle.c``: a plain, slow, FP64 restatement of the AlGDock BPMF hot path
(arXiv:1507.03703), written to check the CUDA library against.  Only the tests, the package's
smoke check and the benchmark's CPU-baseline leg may import this module; the product path never
does.  It shares no code with the CUDA library.  ``build()`` compiles ``oracle.c`` with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Own copies of the unit conventions (A, kcal/mol, amu, fs).
KB = 0.0019872043                      # kcal/(mol K)
K_RESTRAINT = 10000.0 / 4.184 / 100.0  # 10000 kJ/(mol nm^2) in kcal/(mol A^2), Eq. (binding_site)
D0 = 6.0                               # A, binding-site radius
VMAX_R = 10.0 / 4.184                  # soft repulsive cap: 10 kJ/mol per unit scale factor, in kcal/mol

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (portable C11, no intrinsics)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    L.oracle_philox4x32_10.argtypes = [_u32, _u32, _u32]
    L.oracle_u53.argtypes = [C.c_uint32, C.c_uint32]
    L.oracle_u53.restype = C.c_double
    L.oracle_grid_points.argtypes = [C.c_int, _d, _d, _d, _d, C.c_int64, _d, _d, _d, _d, C.c_int]
    L.oracle_grid_points.restype = C.c_int
    L.oracle_grid_direct_sum.argtypes = [C.c_int, _d, _d, _d, _d, _d, C.c_double, _i, _d, _d, _d, C.c_int]
    L.oracle_grid_direct_sum.restype = C.c_int
    L.oracle_soft_elec_cap.argtypes = [C.c_double, C.c_int, _d, _d, _d]
    L.oracle_soft_elec_cap.restype = C.c_double
    L.oracle_prepare_lattices.argtypes = [C.c_int64, _d, _d, C.c_double, C.c_double, _d, _d, _d]
    L.oracle_interp.argtypes = [_d, _i, _d, C.c_double, _d, C.POINTER(C.c_double), _d]
    L.oracle_alpha_sg.argtypes = [C.c_double]
    L.oracle_alpha_sg.restype = C.c_double
    L.oracle_alpha_g.argtypes = [C.c_double]
    L.oracle_alpha_g.restype = C.c_double
    L.oracle_beta.argtypes = [C.c_double]
    L.oracle_beta.restype = C.c_double
    L.oracle_system_create.argtypes = [
        _i, _d, C.c_double, _d, _d, _d, C.c_double, C.c_double, _d, C.c_double, C.c_double,
        C.c_int, _d, _d, _d, _d, C.c_int, _i, _d, _d, C.c_int, _i, _d, _d, C.c_int, _i, _d, _d,
        C.c_int, _d, _d, _d]
    L.oracle_system_create.restype = C.c_void_p
    L.oracle_system_destroy.argtypes = [C.c_void_p]
    L.oracle_system_npairs.argtypes = [C.c_void_p]
    L.oracle_system_npairs.restype = C.c_int
    L.oracle_system_pairs.argtypes = [C.c_void_p, _i, _d, _d]
    L.oracle_state_weights.argtypes = [C.c_void_p, _d, _d, _d]
    L.oracle_grid_terms.argtypes = [C.c_void_p, _d, _d, C.c_void_p, C.c_void_p]
    L.oracle_restraint.argtypes = [C.c_void_p, _d, C.c_void_p]
    L.oracle_restraint.restype = C.c_double
    L.oracle_ligand_ff.argtypes = [C.c_void_p, _d, C.c_void_p, C.c_void_p]
    L.oracle_ligand_ff.restype = C.c_double
    L.oracle_energy_force.argtypes = [C.c_void_p, _d, C.c_double, C.c_double, C.c_void_p, _d]
    L.oracle_vv.argtypes = [C.c_void_p, _d, _d, C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p]
    L.oracle_hmc.argtypes = [C.c_void_p, C.c_int64, _i, C.c_int64, _d, _d, _d, _u8, C.c_int, C.c_uint64,
                             C.c_uint64, C.c_int]
    L.oracle_hmc.restype = C.c_int
    L.oracle_exchange.argtypes = [C.c_int, C.c_int, _d, _d, _d, _i, C.c_int, C.c_int, C.c_uint64,
                                  C.c_uint64, C.c_int64, _i64, _i64]
    L.oracle_reduced_energies.argtypes = [C.c_void_p, C.c_int64, _d, C.c_void_p, C.c_void_p]
    L.oracle_ukn_from_comps.argtypes = [C.c_int, _d, _d, C.c_int64, _d, _d]
    L.oracle_mbar.argtypes = [C.c_int, C.c_int64, _d, _i64, C.c_double, C.c_int, _d]
    L.oracle_mbar.restype = C.c_int
    L.oracle_statistical_inefficiency.argtypes = [C.c_int64, _d]
    L.oracle_statistical_inefficiency.restype = C.c_double
    _lib = L
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ primitives
def philox4x32_10(ctr, key):
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def u53(a: int, b: int) -> float:
    return _load().oracle_u53(a, b)


def alpha_sg(a: float) -> float:
    return _load().oracle_alpha_sg(float(a))


def alpha_g(a: float) -> float:
    return _load().oracle_alpha_g(float(a))


def beta(T: float) -> float:
    return _load().oracle_beta(float(T))


def grid_points(receptor, pts, n_threads: int = 0):
    pts = _f64(pts).reshape(-1, 3)
    n = pts.shape[0]
    ljr, lja, elec = np.empty(n), np.empty(n), np.empty(n)
    _load().oracle_grid_points(receptor.n_atoms, _f64(receptor.xyz), _f64(receptor.rstar), _f64(receptor.eps),
                               _f64(receptor.charge), n, pts, ljr, lja, elec, n_threads)
    return ljr, lja, elec


def grid_direct_sum(receptor, grid, n_threads: int = 0):
    """Raw (untransformed) LJr, LJa and elec grids, each [nz, ny, nx] float64."""
    nx, ny, nz = grid.n
    out = [np.empty(nx * ny * nz) for _ in range(3)]
    _load().oracle_grid_direct_sum(receptor.n_atoms, _f64(receptor.xyz), _f64(receptor.rstar),
                                   _f64(receptor.eps), _f64(receptor.charge), _f64(grid.origin),
                                   float(grid.spacing), np.array(grid.n, dtype=np.int32), out[0], out[1],
                                   out[2], n_threads)
    return tuple(o.reshape(nz, ny, nx) for o in out)


def soft_elec_cap(ligand, vmax_r: float = VMAX_R) -> float:
    return _load().oracle_soft_elec_cap(vmax_r, ligand.n_atoms, _f64(ligand.rstar), _f64(ligand.eps),
                                        _f64(ligand.charge))


def prepare_lattices(ljr, elec, vmax_r, vmax_e):
    shp = np.shape(ljr)
    ljr, elec = _f64(ljr).ravel(), _f64(elec).ravel()
    a, b, c = np.empty_like(ljr), np.empty_like(ljr), np.empty_like(ljr)
    _load().oracle_prepare_lattices(ljr.size, ljr, elec, vmax_r, vmax_e, a, b, c)
    return a.reshape(shp), b.reshape(shp), c.reshape(shp)


def interp(L, grid, x):
    v = C.c_double()
    g = np.zeros(3)
    _load().oracle_interp(_f64(L).ravel(), np.array(grid.n, dtype=np.int32), _f64(grid.origin),
                          float(grid.spacing), _f64(x), C.byref(v), g)
    return v.value, g


class OracleSystem:
    """Lattices + ligand + restraint + one state table (the oracle's own copy of each)."""

    def __init__(self, grid, ljr, lja, elec, ligand, T, alpha, dt_fs, site=None, vmax_r=VMAX_R,
                 vmax_e=None, k_rest=K_RESTRAINT, d0=D0):
        L = _load()
        self._L = L
        self.ligand = ligand
        self.na = ligand.n_atoms
        if vmax_e is None:
            vmax_e = soft_elec_cap(ligand, vmax_r)
        self.vmax_e = vmax_e
        site = grid.center if site is None else site
        self.T, self.alpha, self.dt = _f64(T), _f64(alpha), _f64(dt_fs)
        self.K = int(self.T.size)
        lg = ligand
        self._keep = [_f64(ljr).ravel(), _f64(lja).ravel(), _f64(elec).ravel()]
        self.h = L.oracle_system_create(
            np.array(grid.n, dtype=np.int32), _f64(grid.origin), float(grid.spacing), self._keep[0],
            self._keep[1], self._keep[2], float(vmax_r), float(vmax_e), _f64(site), float(k_rest), float(d0),
            self.na, _f64(lg.mass), _f64(lg.charge), _f64(lg.rstar), _f64(lg.eps), lg.bonds.shape[0],
            _i32(lg.bonds), _f64(lg.bond_k), _f64(lg.bond_r0), lg.angles.shape[0], _i32(lg.angles),
            _f64(lg.angle_k), _f64(lg.angle_theta0), lg.torsions.shape[0], _i32(lg.torsions),
            _f64(lg.torsion_V), _f64(lg.torsion_gamma), self.K, self.T, self.alpha, self.dt)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._L.oracle_system_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def pairs(self):
        n = self._L.oracle_system_npairs(self.h)
        p, sl, se = np.zeros((max(n, 1), 2), dtype=np.int32), np.zeros(max(n, 1)), np.zeros(max(n, 1))
        self._L.oracle_system_pairs(self.h, p, sl, se)
        return p[:n], sl[:n], se[:n]

    def state_weights(self):
        a, b, c = np.zeros(self.K), np.zeros(self.K), np.zeros(self.K)
        self._L.oracle_state_weights(self.h, a, b, c)
        return a, b, c

    def grid_terms(self, x):
        x = _f64(x)
        psi = np.zeros(2)
        gs, gg = np.zeros(x.size), np.zeros(x.size)
        self._L.oracle_grid_terms(self.h, x, psi, _ptr(gs), _ptr(gg))
        return psi, gs.reshape(-1, 3), gg.reshape(-1, 3)

    def restraint(self, x):
        x = _f64(x)
        F = np.zeros(x.size)
        e = self._L.oracle_restraint(self.h, x, _ptr(F))
        return e, F.reshape(-1, 3)

    def ligand_ff(self, x):
        x = _f64(x)
        F = np.zeros(x.size)
        terms = np.zeros(4)
        e = self._L.oracle_ligand_ff(self.h, x, _ptr(F), _ptr(terms))
        return e, F.reshape(-1, 3), terms

    def energy_force(self, x, w_sg=0.0, w_g=0.0):
        """Components {U_L, U_I, Psi_sg, Psi_g} and the force of grid weights (w_sg, w_g)."""
        x = _f64(x)
        F = np.zeros(x.size)
        comps = np.zeros(4)
        self._L.oracle_energy_force(self.h, x, float(w_sg), float(w_g), _ptr(F), comps)
        return comps, F.reshape(-1, 3)

    def vv(self, x, v, w_sg, w_g, dt, n_steps):
        """Velocity Verlet at fixed weights.  Returns (x, v, H[0..n_steps])."""
        x = np.array(x, dtype=np.float64, order="C")
        v = np.array(v, dtype=np.float64, order="C")
        H = np.zeros(n_steps + 1)
        self._L.oracle_vv(self.h, x, v, float(w_sg), float(w_g), float(dt), int(n_steps), _ptr(H))
        return x, v, H

    def hmc(self, x, state_of, n_steps, seed, cycle, rep_offset=0, n_threads=0):
        """One HMC trial per replica (in place on a float64 copy).  Returns
        (x_new, comps [R,4], dH [R], accepted [R] uint8, threads used)."""
        x = np.array(x, dtype=np.float64, order="C").reshape(-1, self.na, 3)
        R = x.shape[0]
        comps, dH, acc = np.zeros((R, 4)), np.zeros(R), np.zeros(R, dtype=np.uint8)
        nt = self._L.oracle_hmc(self.h, R, _i32(state_of), int(rep_offset), x, comps, dH, acc, int(n_steps),
                                int(seed), int(cycle), int(n_threads))
        return x, comps, dH, acc, nt

    def reduced_energies(self, x):
        x = _f64(x).reshape(-1, self.na, 3)
        N = x.shape[0]
        u = np.zeros((self.K, N))
        comps = np.zeros((N, 4))
        self._L.oracle_reduced_energies(self.h, N, x, _ptr(u), _ptr(comps))
        return u, comps


def exchange(T, alpha, comps, config_of, n_sweeps, max_sep, seed, cycle, ladder_offset=0):
    """Replica-exchange sweeps on each ladder.  comps [L, K, 4], config_of [L, K] int32 (copied).
    Returns (config_of_new, attempts [max_sep, K], accepts [max_sep, K])."""
    comps = _f64(comps)
    L_, K = comps.shape[0], comps.shape[1]
    cfg = np.array(config_of, dtype=np.int32, order="C").reshape(L_, K)
    att = np.zeros((max_sep, K), dtype=np.int64)
    acc = np.zeros((max_sep, K), dtype=np.int64)
    _load().oracle_exchange(L_, K, _f64(T), _f64(alpha), comps, cfg, int(n_sweeps), int(max_sep), int(seed),
                            int(cycle), int(ladder_offset), att, acc)
    return cfg, att, acc


def ukn_from_comps(T, alpha, comps):
    comps = _f64(comps).reshape(-1, 4)
    T = _f64(T)
    u = np.zeros((T.size, comps.shape[0]))
    _load().oracle_ukn_from_comps(T.size, T, _f64(alpha), comps.shape[0], comps, u)
    return u


def mbar(u_kn, N_k, tol=1e-10, max_iter=10000):
    """Returns (f_k, iterations); iterations = -1 if not converged."""
    u_kn = _f64(u_kn)
    K, N = u_kn.shape
    f = np.zeros(K)
    it = _load().oracle_mbar(K, N, u_kn, np.ascontiguousarray(N_k, dtype=np.int64), float(tol), int(max_iter), f)
    return f, it


def mbar_partials(u_kn, N_k, f):
    """The state sums of one MBAR iteration over a subset of the samples (Shirts & Chodera 2008, as
    cited in "Estimation"): in f_i = -ln sum_n exp(-u_in) / D_n with
    D_n = sum_k N_k exp(f_k - u_kn), the sum over n splits over any partition of the samples, while
    D_n belongs to its own sample.  For the columns given, returns [K][2] pairs (M_i, S_i) with
    sum_n exp(-u_in - ln D_n) = S_i exp(M_i) (M_i = -inf, S_i = 0 without samples).  N_k are the
    counts over all samples.  FP64, numpy."""
    u = np.asarray(u_kn, dtype=np.float64)
    K = u.shape[0]
    out = np.zeros((K, 2))
    out[:, 0] = -np.inf
    if u.shape[1] == 0:
        return out
    lw = np.log(np.asarray(N_k, dtype=np.float64))[:, None] + np.asarray(f, dtype=np.float64)[:, None] - u
    c = lw.max(axis=0)
    log_d = c + np.log(np.exp(lw - c).sum(axis=0))
    a = -u - log_d[None, :]
    m = a.max(axis=1)
    out[:, 0] = m
    out[:, 1] = np.exp(a - m[:, None]).sum(axis=1)
    return out


def statistical_inefficiency(a):
    a = _f64(a)
    return _load().oracle_statistical_inefficiency(a.size, a)


def bpmf_kT(f_bc, f_cd):
    """beta_T B = f_BC,L + f'_CD, each the last-minus-first free energy of its ladder (Estimation)."""
    return (f_bc[-1] - f_bc[0]) + (f_cd[-1] - f_cd[0])


def run_ladder(osys, x0, n_chains, n_cycles, n_steps, seed, n_sweeps=25, max_sep=5, rep_offset=0,
               ladder_offset=0, burn_in=0, n_threads=0, n_external=0):
    """Replica-exchange HMC on one ladder (the oracle's own driver of the sampling loop).

    Slot r = c*K + i holds one configuration of chain c; config_of[c, k] is the slot index (within
    the chain) of the configuration at state k.  Each cycle ("Equilibration and production"): one
    HMC trial per slot at its state, then ``n_external`` external-coordinate moves of every slot
    whose state has alpha < 0.01 ("Sampling"; 0: none), then ``n_sweeps`` exchange sweeps per
    chain.  After ``burn_in`` cycles every slot's components are recorded with its state.  Returns
    (comps [S, 4], state [S], acceptance per state [K], exchange accepts / attempts [max_sep, K],
    final x).
    """
    K = osys.K
    x = np.array(x0, dtype=np.float64).reshape(n_chains * K, osys.na, 3)
    config_of = np.tile(np.arange(K, dtype=np.int32), (n_chains, 1))
    samples, states = [], []
    hmc_acc = np.zeros(K)
    hmc_n = np.zeros(K)
    ex_att = np.zeros((max_sep, K), dtype=np.int64)
    ex_acc = np.zeros((max_sep, K), dtype=np.int64)
    for cyc in range(n_cycles):
        state_of = np.empty(n_chains * K, dtype=np.int32)
        for c in range(n_chains):
            state_of[c * K + config_of[c]] = np.arange(K, dtype=np.int32)
        x, comps, dH, acc, _ = osys.hmc(x, state_of, n_steps, seed, cyc, rep_offset=rep_offset,
                                        n_threads=n_threads)
        if n_external > 0:
            x, comps, _ = osys.external_moves(x, comps, state_of, n_external, seed, cyc, rep_offset=rep_offset)
        np.add.at(hmc_acc, state_of, acc)
        np.add.at(hmc_n, state_of, 1)
        config_of, att, ac = exchange(osys.T, osys.alpha, comps.reshape(n_chains, K, 4), config_of, n_sweeps,
                                      max_sep, seed, cyc, ladder_offset=ladder_offset)
        ex_att += att
        ex_acc += ac
        if cyc >= burn_in:
            st = np.empty(n_chains * K, dtype=np.int32)
            for c in range(n_chains):
                st[c * K + config_of[c]] = np.arange(K, dtype=np.int32)
            samples.append(comps.copy())
            states.append(st)
    comps = np.concatenate(samples, 0) if samples else np.zeros((0, 4))
    states = np.concatenate(states, 0) if states else np.zeros(0, dtype=np.int32)
    return comps, states, hmc_acc / np.maximum(hmc_n, 1), (ex_acc, ex_att), x


def ladder_free_energies(T, alpha, comps, states, tol=1e-10, max_iter=10000):
    """MBAR over all recorded samples of one ladder; f_k with f_0 = 0."""
    K = len(T)
    order = np.argsort(states, kind="stable")
    u = ukn_from_comps(T, alpha, comps[order])
    N_k = np.bincount(states, minlength=K).astype(np.int64)
    return mbar(u, N_k, tol=tol, max_iter=max_iter)


# ------------------------------------------------------------------ learned pose proposal
NFEAT, NHID, NCOMP, DMAX, NOUT = 64, 256, 8, 22, 8 * (1 + 2 * 22)
_MLP_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def _learned_sigs(L):
    if getattr(L, "_learned", False):
        return
    L.oracle_set_bf16_activations.argtypes = [C.c_int]
    L.oracle_learned_ntorsions.argtypes = [C.c_void_p]
    L.oracle_learned_ntorsions.restype = C.c_int
    L.oracle_features.argtypes = [C.c_void_p, _d, _d, C.c_int, _d]
    L.oracle_apply.argtypes = [C.c_void_p, _d, _d, _d]
    L.oracle_pose_delta.argtypes = [C.c_void_p, _d, _d, _d]
    L.oracle_mlp_forward.argtypes = [_d] * 8 + [C.c_int, _d, _d, C.c_void_p, C.c_void_p, C.c_void_p]
    L.oracle_mlp_backward.argtypes = [_d, _d, _d, C.c_int, _d, _d, _d, _d, _d] + [_d] * 8
    L.oracle_mixture_logq.argtypes = [_d, C.c_int, _d, C.c_void_p]
    L.oracle_mixture_logq.restype = C.c_double
    L.oracle_mixture_sample.argtypes = [_d, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, _d]
    L.oracle_learned_mh.argtypes = ([C.c_void_p] + [_d] * 8 + [C.c_int64, _i, C.c_int64, _d, _d, C.c_int, C.c_int,
                                    C.c_uint64, C.c_uint64, _i, C.c_void_p])
    L._learned = True


def _p(params):
    return [_f64(params[k]).ravel() for k in _MLP_KEYS]


def set_bf16_activations(on: bool):
    """Round the network's input and hidden activations to BF16 (as a BF16 tensor-core
    implementation stores them) in every later forward pass; default off (FP64)."""
    L = _load()
    _learned_sigs(L)
    L.oracle_set_bf16_activations(1 if on else 0)


def mlp_forward(params, X):
    """FP64 forward pass: returns (out [B, 360], h1, h2, h3)."""
    L = _load()
    _learned_sigs(L)
    X = _f64(X).reshape(-1, NFEAT)
    B = X.shape[0]
    out, h1, h2, h3 = np.zeros((B, NOUT)), np.zeros((B, NHID)), np.zeros((B, NHID)), np.zeros((B, NHID))
    L.oracle_mlp_forward(*_p(params), B, X, out, _ptr(h1), _ptr(h2), _ptr(h3))
    return out, h1, h2, h3


def mlp_backward(params, X, h1, h2, h3, dout):
    """Gradients of sum <dout, out> with respect to every parameter (dict like params)."""
    L = _load()
    _learned_sigs(L)
    X = _f64(X).reshape(-1, NFEAT)
    B = X.shape[0]
    g = {k: np.zeros_like(_f64(params[k])) for k in _MLP_KEYS}
    L.oracle_mlp_backward(_f64(params["W2"]).ravel(), _f64(params["W3"]).ravel(), _f64(params["W4"]).ravel(), B, X,
                          _f64(h1), _f64(h2), _f64(h3), _f64(dout), *[g[k] for k in _MLP_KEYS])
    return g


def mixture_logq(o, D, delta, grad=False):
    L = _load()
    _learned_sigs(L)
    g = np.zeros(NOUT) if grad else None
    lq = L.oracle_mixture_logq(_f64(o), int(D), _f64(np.resize(np.asarray(delta, dtype=np.float64), DMAX)), _ptr(g))
    return (lq, g) if grad else lq


def mixture_sample(o, D, seed, rep, ctr):
    L = _load()
    _learned_sigs(L)
    out = np.zeros(DMAX)
    L.oracle_mixture_sample(_f64(o), int(D), int(seed), int(rep), int(ctr), out)
    return out[:D]


class _LearnedMixin:
    def learned_ntorsions(self):
        _learned_sigs(self._L)
        return self._L.oracle_learned_ntorsions(self.h)

    def features(self, x, comps, k):
        _learned_sigs(self._L)
        f = np.zeros(NFEAT)
        self._L.oracle_features(self.h, _f64(x).ravel(), _f64(comps), int(k), f)
        return f

    def apply(self, x, delta):
        _learned_sigs(self._L)
        y = np.zeros(3 * self.na)
        d = np.zeros(DMAX)
        d[:len(delta)] = delta
        self._L.oracle_apply(self.h, _f64(x).ravel(), d, y)
        return y.reshape(-1, 3)

    def pose_delta(self, x, y):
        _learned_sigs(self._L)
        d = np.zeros(DMAX)
        self._L.oracle_pose_delta(self.h, _f64(x).ravel(), _f64(y).ravel(), d)
        return d[:6 + self.learned_ntorsions()]

    def learned_mh(self, params, x, comps, state_of, n_moves, seed, cycle, rep_offset=0, n_torsions=-1):
        """n_moves learned proposals per replica (moving the first n_torsions torsions; negative: all).
        Returns (x, comps, accepts [R], last log-ratio [R])."""
        _learned_sigs(self._L)
        x = np.array(x, dtype=np.float64, order="C").reshape(-1, self.na, 3)
        comps = np.array(comps, dtype=np.float64, order="C").reshape(-1, 4)
        R = x.shape[0]
        acc = np.zeros(R, dtype=np.int32)
        lr = np.zeros(R)
        self._L.oracle_learned_mh(self.h, *_p(params), R, _i32(state_of), int(rep_offset), x, comps, int(n_moves),
                                  int(n_torsions), int(seed), int(cycle), acc, _ptr(lr))
        return x, comps, acc, lr


for _name in ("learned_ntorsions", "features", "apply", "pose_delta", "learned_mh"):
    setattr(OracleSystem, _name, getattr(_LearnedMixin, _name))


# ------------------------------------------------------------------ external-coordinate moves
SIGMA_TRANSLATION = 0.6   # A per dimension ("Sampling")
ALPHA_MAX_EXTERNAL = 0.01  # moves only below this alpha ("Sampling")


def _external_sigs(L):
    if getattr(L, "_external", False):
        return
    L.oracle_random_rotation.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, _d]
    L.oracle_external_moves.argtypes = [C.c_void_p, C.c_int64, _i, C.c_int64, _d, _d, C.c_int, C.c_double,
                                        C.c_double, C.c_uint64, C.c_uint64, _i, C.c_void_p]
    L._external = True


def random_rotation(a, b, c):
    """Rotation matrix (3x3) of the quaternion built from three 32-bit words (Shoemake)."""
    L = _load()
    _external_sigs(L)
    R = np.zeros(9)
    L.oracle_random_rotation(int(a) & 0xFFFFFFFF, int(b) & 0xFFFFFFFF, int(c) & 0xFFFFFFFF, R)
    return R.reshape(3, 3)


def _external_moves(self, x, comps, state_of, n_moves, seed, cycle, rep_offset=0, alpha_max=ALPHA_MAX_EXTERNAL,
                    sigma=SIGMA_TRANSLATION, logratio=False):
    """n_moves external-coordinate moves per replica whose state has alpha < alpha_max.
    Returns (x, comps, accepts [R]); with logratio=True also the last move's log acceptance
    ratio [R]."""
    _external_sigs(self._L)
    x = np.array(x, dtype=np.float64, order="C").reshape(-1, self.na, 3)
    comps = np.array(comps, dtype=np.float64, order="C").reshape(-1, 4)
    R = x.shape[0]
    acc = np.zeros(R, dtype=np.int32)
    lr = np.zeros(R) if logratio else None
    self._L.oracle_external_moves(self.h, R, _i32(state_of), int(rep_offset), x, comps, int(n_moves),
                                  float(alpha_max), float(sigma), int(seed), int(cycle), acc, _ptr(lr))
    return (x, comps, acc, lr) if logratio else (x, comps, acc)


OracleSystem.external_moves = _external_moves


# ------------------------------------------------------------------ equilibration detection
def detect_equilibration(a, stride=1, n_cand=None):
    """Candidates t0 = c * stride: (g of each tail [n_cand], best t0, its N_eff = (T - t0) / g)."""
    L = _load()
    if not getattr(L, "_equil", False):
        L.oracle_detect_equilibration.argtypes = [C.c_int64, _d, C.c_int64, C.c_int, _d,
                                                  C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L._equil = True
    a = _f64(a).ravel()
    T = a.size
    if n_cand is None:
        n_cand = (T - 2) // stride + 1
    g = np.zeros(n_cand)
    t0 = C.c_int64(0)
    ne = C.c_double(0.0)
    L.oracle_detect_equilibration(T, a, int(stride), int(n_cand), g, C.byref(t0), C.byref(ne))
    return g, int(t0.value), float(ne.value)


# ------------------------------------------------------------------ protocol initialization
def _protocol_sigs(L):
    if getattr(L, "_protocol", False):
        return
    L.oracle_system_set_states.argtypes = [C.c_void_p, C.c_int, _d, _d, _d]
    L.oracle_state_statistics.argtypes = [C.c_void_p, C.c_int64, _d, C.c_int, _d]
    L.oracle_next_temperature.argtypes = [C.c_double] * 4
    L.oracle_next_temperature.restype = C.c_double
    L.oracle_next_alpha.argtypes = [C.c_double] * 7
    L.oracle_next_alpha.restype = C.c_double
    L.oracle_resample.argtypes = [C.c_int64, _d, C.c_int, C.c_uint64, C.c_uint32, np.ctypeslib.ndpointer(
        dtype=np.int64, flags="C_CONTIGUOUS")]
    L.oracle_mean_pacc.argtypes = [C.c_void_p, C.c_int64, _d, _d, C.c_int, C.c_int]
    L.oracle_mean_pacc.restype = C.c_double
    L.oracle_adapt_dt.argtypes = [C.c_double, C.c_double]
    L.oracle_adapt_dt.restype = C.c_double
    L._protocol = True


def next_temperature(T, sigma_U, speed, T_end=600.0):
    L = _load()
    _protocol_sigs(L)
    return L.oracle_next_temperature(float(T), float(sigma_U), float(speed), float(T_end))


def next_alpha(alpha, sigma_sg, sigma_g, sigma_u, speed, T_T=300.0, T_H=600.0):
    L = _load()
    _protocol_sigs(L)
    return L.oracle_next_alpha(float(alpha), float(sigma_sg), float(sigma_g), float(sigma_u), float(speed),
                               float(T_T), float(T_H))


def resample(logw, n_out, seed, ctr):
    """Indices of n_out importance-resampled draws (weights exp(logw))."""
    L = _load()
    _protocol_sigs(L)
    logw = _f64(logw).ravel()
    idx = np.zeros(int(n_out), dtype=np.int64)
    L.oracle_resample(logw.size, logw, int(n_out), int(seed), int(ctr) & 0xFFFFFFFF, idx)
    return idx


def adapt_dt(dt, acc):
    L = _load()
    _protocol_sigs(L)
    return L.oracle_adapt_dt(float(dt), float(acc))


def _set_states(self, T, alpha, dt):
    _protocol_sigs(self._L)
    self.T, self.alpha, self.dt = _f64(T), _f64(alpha), _f64(dt)
    self.K = int(self.T.size)
    self._L.oracle_system_set_states(self.h, self.K, self.T, self.alpha, self.dt)


def _state_statistics(self, comps, k):
    """{sigma[U_L + U_I], sigma[Psi_sg], sigma[Psi_g], sigma[u_k]} over the samples comps [n][4]."""
    _protocol_sigs(self._L)
    c = _f64(comps).reshape(-1, 4)
    out = np.zeros(4)
    self._L.oracle_state_statistics(self.h, c.shape[0], c, int(k), out)
    return out


def _mean_pacc(self, comps_a, comps_b, ka, kb):
    _protocol_sigs(self._L)
    a, b = _f64(comps_a).reshape(-1, 4), _f64(comps_b).reshape(-1, 4)
    return self._L.oracle_mean_pacc(self.h, a.shape[0], a, b, int(ka), int(kb))


OracleSystem.set_states = _set_states
OracleSystem.state_statistics = _state_statistics
OracleSystem.mean_pacc = _mean_pacc


def _sample_state(osys, k, seeds, n_trials, n_steps, seed, cycle0, max_attempts=20):
    """Sampling and adaptation at state k: n_trials HMC trials from the seeds; the time step is
    adapted (and the run repeated from the seeds) until the acceptance lies in [0.4, 0.8].
    Returns (comps [n_trials * n_seeds, 4], x [same, na, 3], acceptance, dt, next cycle)."""
    dt = float(osys.dt[k])
    cycle = cycle0
    for _ in range(max_attempts):
        x = np.array(seeds, dtype=np.float64)
        st = np.full(x.shape[0], k, dtype=np.int32)
        cs, xs, acc = [], [], 0
        for t in range(n_trials):
            x, c, _, a, _ = osys.hmc(x, st, n_steps, seed, cycle)
            cycle += 1
            cs.append(c)
            xs.append(x.copy())
            acc += int(a.sum())
        rate = acc / (n_trials * x.shape[0])
        if 0.4 <= rate <= 0.8:
            break
        new = adapt_dt(dt, rate)
        if new == dt:
            break
        dt = new
        dts = osys.dt.copy()
        dts[k] = dt
        osys.set_states(osys.T, osys.alpha, dts)
    return np.concatenate(cs), np.concatenate(xs), rate, dt, cycle


def build_leg(osys, leg, seeds, seed, speed=None, n_trials=40, n_steps=50, T_T=300.0, T_H=600.0, dt0=2.0,
              max_states=400, max_reselect=40):
    """"Initialization" of one leg, state after state: sampling and time-step adaptation at the
    current state, the next state's parameter one thermodynamic-length step away (warming leg:
    T; coupling leg: alpha), seeds resampled from the current state with weights exp(u_k - u_next),
    sampling at the candidate, and the check on the mean exchange probability (below 0.4: the speed
    shrinks by 4/5 and the candidate is placed again; above 0.99: the current state is dropped).
    Returns dict(T, alpha, dt, pacc [neighbours], acceptance, speed)."""
    bc = leg == "bc"
    speed = (20.0 if bc else 0.2) if speed is None else float(speed)
    T, A, D = ([T_T], [np.nan], [dt0]) if bc else ([T_H], [0.0], [dt0])
    osys.set_states(T, A, D)
    cycle = 0
    comps_k, x_k, rate, dt, cycle = _sample_state(osys, 0, seeds, n_trials, n_steps, seed, cycle)
    D[0] = dt
    pacc, rates = [], [rate]
    for _ in range(max_states):
        k = len(T) - 1
        if (bc and T[k] >= 600.0) or (not bc and A[k] >= 1.0):
            break
        sig = osys.state_statistics(comps_k, k)
        for tries in range(max_reselect):
            if bc:
                Tn, An = next_temperature(T[k], sig[0], speed, 600.0), np.nan
            else:
                An = next_alpha(A[k], sig[1], sig[2], sig[3], speed, T_T, T_H)
                Tn = (T_T - T_H) * An + T_H
            osys.set_states(T + [Tn], A + [An], D + [D[k]])
            u = ukn_from_comps(osys.T, osys.alpha, comps_k)
            logw = u[k] - u[k + 1]
            pick = resample(logw, seeds.shape[0], seed, 1_000_000 + cycle)
            comps_n, x_n, rate_n, dt_n, cycle = _sample_state(osys, k + 1, x_k[pick], n_trials, n_steps, seed, cycle)
            p = osys.mean_pacc(comps_k, comps_n, k, k + 1)
            if p >= 0.4:
                break
            speed *= 0.8
        if p > 0.99 and k > 0:  # state k is too close to its successor: the successor replaces it
            T[k], A[k], D[k] = Tn, An, dt_n
            osys.set_states(T, A, D)
            pacc[-1] = osys.mean_pacc(prev_comps, comps_n, k - 1, k)
        else:
            T.append(Tn)
            A.append(An)
            D.append(dt_n)
            pacc.append(p)
        rates.append(rate_n)
        prev_comps = comps_k
        comps_k, x_k = comps_n, x_n
        osys.set_states(T, A, D)
    return {"T": np.array(T), "alpha": np.array(A), "dt": np.array(D), "pacc": np.array(pacc),
            "acceptance": np.array(rates), "speed": speed}


# ------------------------------------------------------------------ end points: target force field and FEP
def target_interaction(receptor, ligand, x, n_threads: int = 0):
    """Receptor-ligand energy of the target force field, computed directly at the ligand atoms'
    positions ("Thermodynamic Cycle": the target force field evaluates receptor-ligand
    interactions directly, the sampling force field by grid interpolation).  x: [N, n_atoms, 3];
    returns [N] float64 (kcal/mol)."""
    L = _load()
    if not getattr(L, "_target", False):
        L.oracle_target_interaction.argtypes = [C.c_int, _d, _d, _d, _d, C.c_int, _d, _d, _d, C.c_int64, _d, _d,
                                                C.c_int]
        L.oracle_target_interaction.restype = C.c_int
        L._target = True
    x = _f64(x).reshape(-1, ligand.n_atoms, 3)
    out = np.empty(x.shape[0])
    L.oracle_target_interaction(receptor.n_atoms, _f64(receptor.xyz), _f64(receptor.rstar), _f64(receptor.eps),
                                _f64(receptor.charge), ligand.n_atoms, _f64(ligand.rstar), _f64(ligand.eps),
                                _f64(ligand.charge), x.shape[0], x, out, n_threads)
    return out


def fep(du):
    """Zwanzig free energy perturbation ("Estimation": f_AB and f_DE by free energy perturbation)
    from reduced energy differences du_n = beta (U_target - U_sampling) of N samples drawn in the
    sampling state:  f = -ln (1/N) sum_n exp(-du_n).

    Also returns the Kish effective sample size n_eff = (sum w)^2 / sum w^2 of the weights
    w_n = exp(-du_n), the first-order (delta-method) standard error of f for independent samples,
    sigma^2 = var(w) / (N mean(w)^2) = (N / n_eff - 1) / (N - 1), and the smallest du.
    The weights are taken relative to the smallest du, which leaves f unchanged."""
    import math
    du = np.asarray(du, dtype=np.float64).reshape(-1)
    N = du.shape[0]
    if N == 0:
        raise ValueError("fep needs at least one sample")
    m = float(du.min())
    w = np.exp(-(du - m))
    s1 = math.fsum(w)
    s2 = math.fsum(w * w)
    f = m - math.log(s1 / N)
    n_eff = s1 * s1 / s2
    sigma = math.sqrt(max(N / n_eff - 1.0, 0.0) / (N - 1)) if N > 1 else math.nan
    return {"f": f, "sigma": sigma, "n_eff": n_eff, "du_min": m}


# ------------------------------------------------------------------ state insertion between cycles
def split_ladder(T, alpha, dt, attempts, accepts, threshold=0.4, T_T=300.0, T_H=600.0):
    """The between-cycle insertion rule ("Equilibration and production"): wherever the mean
    replica-exchange acceptance between neighbouring states a and a+1 over the cycle fell below
    the threshold (0.4), one state is placed between them.  Its parameters are the midpoint of
    the leg's control parameter: the geometric mean of the temperatures on the warming leg (alpha
    NaN, geometric temperatures), the mean alpha on the coupling leg with T = T_H + (T_T - T_H)
    alpha; its time step is the smaller of the two.  attempts / accepts hold the neighbour-pair
    counts [K - 1].  Returns (T, alpha, dt, inserted) with inserted the new states' indices in
    the returned ladder."""
    T, alpha, dt = list(map(float, T)), list(map(float, alpha)), list(map(float, dt))
    K = len(T)
    split = [a for a in range(K - 1) if attempts[a] > 0 and accepts[a] / attempts[a] < threshold]
    oT, oA, oD, inserted = [], [], [], []
    for k in range(K):
        oT.append(T[k])
        oA.append(alpha[k])
        oD.append(dt[k])
        if k in split:
            if alpha[k] != alpha[k]:  # NaN: the warming leg
                newT, newA = (T[k] * T[k + 1]) ** 0.5, float("nan")
            else:
                newA = 0.5 * (alpha[k] + alpha[k + 1])
                newT = T_H + (T_T - T_H) * newA
            inserted.append(len(oT))
            oT.append(newT)
            oA.append(newA)
            oD.append(min(dt[k], dt[k + 1]))
    return np.array(oT), np.array(oA), np.array(oD), inserted
