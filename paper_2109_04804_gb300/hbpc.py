"""Thin ctypes binding of libhbpc (C-ABI in include/hbpc.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Device buffers are torch CUDA tensors (PyTorch provides device memory and
streams); host buffers are numpy arrays.  Importing this module loads the
shared library and raises ImportError if it has not been built (there is no
fallback implementation).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhbpc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libhbpc.so is not built; run __graft_entry__.build() "
                      "(or python paper_2109_04804_gb300/build.py) first")
_lib = ctypes.CDLL(LIB_PATH)

# -- enums (hbpc.h) -----------------------------------------------------------
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NO_CONVERGENCE, ERR_NONFINITE, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = range(8)
LAW_ADVECTION, LAW_BURGERS, LAW_EULER, LAW_NAVIER_STOKES = 0, 1, 2, 3
FLUX_GLOBAL_LF, FLUX_RUSANOV = 0, 1
NODES_LOBATTO, NODES_GAUSS = 0, 1
PC_NONE, PC_BJEXT, PC_LEARNED, PC_BJEXT_H = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
BC_PERIODIC, BC_DIRICHLET, BC_WALL, BC_NOSLIP = 0, 1, 2, 3
PC_LOSS = {"probe": 0, "inverse": 1}
PHASES = ("jv", "operator", "arnoldi_dot", "arnoldi_update", "vector", "pc_apply", "pc_build")

STATUS_NAMES = {0: "HBPC_OK", 1: "HBPC_ERR_INVALID_ARG", 2: "HBPC_ERR_OOM", 3: "HBPC_ERR_CUDA",
                4: "HBPC_ERR_NO_CONVERGENCE", 5: "HBPC_ERR_NONFINITE", 6: "HBPC_ERR_TIMEOUT",
                7: "HBPC_ERR_UNSUPPORTED"}


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("periodic", ctypes.c_int)]


def _mesh(dim, n, lo, hi, periodic=1):
    pad = lambda v, fill: (list(v) + [fill] * 3)[:3]
    return Mesh(dim, (ctypes.c_int * 3)(*pad(n, 1)), (ctypes.c_double * 3)(*pad(lo, 0.0)),
                (ctypes.c_double * 3)(*pad(hi, 1.0)), periodic)


class Physics(ctypes.Structure):
    _fields_ = [("law", ctypes.c_int), ("flux", ctypes.c_int), ("a", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("eps", ctypes.c_double), ("lf_scale", ctypes.c_double),
                ("nu", ctypes.c_double), ("eta_br2", ctypes.c_double), ("prandtl", ctypes.c_double)]


class Solver(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("kmax", ctypes.c_int), ("dt", ctypes.c_double),
                ("tol_newton_rel", ctypes.c_double), ("tol_newton_abs", ctypes.c_double),
                ("tol_gmres_rel", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("gmres_max_iter", ctypes.c_int), ("newton_max_iter", ctypes.c_int),
                ("pc", ctypes.c_int), ("precision", ctypes.c_int), ("t_end", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("krylov_blocks", ctypes.c_int), ("krylov_us", ctypes.c_double),
                ("krylov_us_default", ctypes.c_double), ("pc_elems_per_block", ctypes.c_int),
                ("pc_us", ctypes.c_double), ("pc_us_default", ctypes.c_double), ("cooperative_cgs", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("newton_solves", ctypes.c_longlong),
                ("newton_its", ctypes.c_longlong), ("gmres_its", ctypes.c_longlong),
                ("r1_evals", ctypes.c_longlong), ("r2_evals", ctypes.c_longlong),
                ("launches", ctypes.c_longlong), ("t", ctypes.c_double), ("arnoldi_cols", ctypes.c_longlong),
                ("pc_exact_blocks", ctypes.c_longlong), ("pc_apply_tc", ctypes.c_longlong)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_CTX = ctypes.c_void_p

_SIGS = {
    "hbpc_create": (_I, [ctypes.POINTER(_CTX), ctypes.POINTER(Mesh), _I, _I, ctypes.POINTER(Physics),
                         ctypes.POINTER(Solver), _P]),
    "hbpc_destroy": (None, [_CTX]),
    "hbpc_ndof": (ctypes.c_longlong, [_CTX]),
    "hbpc_nvar": (_I, [_CTX]),
    "hbpc_node_coords": (_I, [_CTX, _P]),
    "hbpc_basis": (_I, [_I, _I, _P, _P, _P, _P, _P]),
    "hbpc_set_state": (_I, [_CTX, _P, _I]),
    "hbpc_get_state": (_I, [_CTX, _P, _I]),
    "hbpc_set_time": (_I, [_CTX, _D]),
    "hbpc_step": (_I, [_CTX, _I]),
    "hbpc_advance_to": (_I, [_CTX, _D]),
    "hbpc_run": (_I, [_CTX]),
    "hbpc_set_wait_limit": (_I, [_CTX, _D]),
    "hbpc_set_corrector_batch": (_I, [_CTX, _I]),
    "hbpc_set_schur": (_I, [_CTX, _I]),
    "hbpc_set_boundary": (_I, [_CTX, _I, _I, _P, _I, _P]),
    "hbpc_set_step_graph": (_I, [_CTX, _I]),
    "hbpc_set_pc_rebuild": (_I, [_CTX, _I]),
    "hbpc_eval_R1": (_I, [_CTX, _P, _P]),
    "hbpc_eval_R2": (_I, [_CTX, _P, _P, _P]),
    "hbpc_eval_G": (_I, [_CTX, _P, _D, _D, _P, _P]),
    "hbpc_eval_Jv": (_I, [_CTX, _D, _D, _P, _P, _P]),
    "hbpc_newton_solve": (_I, [_CTX, _P, _D, _D, _P, _P, _P]),
    "hbpc_eval_pc": (_I, [_CTX, _D, _D, _P, _P, _P]),
    "hbpc_set_pc": (_I, [_CTX, _I]),
    "hbpc_pc_model_info": (_I, [_CTX, _P, _P, _P, _P]),
    "hbpc_pc_model_init": (_I, [_CTX, ctypes.c_ulonglong, _D]),
    "hbpc_pc_model_get": (_I, [_CTX, _P]),
    "hbpc_pc_model_set": (_I, [_CTX, _P]),
    "hbpc_pc_loss_grad": (_I, [_CTX, _I, _I, _I, _P, _P, _P, _P, _P, _P]),
    "hbpc_pc_collect": (_I, [_CTX, _I, _I]),
    "hbpc_pc_model_forward": (_I, [_CTX, _I, _P, _P, _P]),
    "hbpc_pc_adam_step": (_I, [_CTX, _P, _D]),
    "hbpc_pc_train": (_I, [_CTX, _I, _I, _I, _I, _D, ctypes.c_ulonglong, _P, _P]),
    "hbpc_fp64_fma_peak": (_I, [ctypes.POINTER(ctypes.c_double)]),
    "hbpc_eval_Jv_noalloc": (_I, [ctypes.POINTER(Mesh), _I, _I, ctypes.POINTER(Physics), _D, _D, _D,
                                  _P, _P, _P, _P]),
    "hbpc_get_stats": (_I, [_CTX, ctypes.POINTER(Stats)]),
    "hbpc_reset_stats": (_I, [_CTX]),
    "hbpc_last_error": (ctypes.c_char_p, [_CTX]),
    "hbpc_profile_enable": (_I, [_CTX, _I]),
    "hbpc_profile_get": (_I, [_CTX, _P, _P, _I]),
    "hbpc_batch_create": (_I, [ctypes.POINTER(_CTX), _I, _P, _P, _I, _P, ctypes.POINTER(Solver), _I]),
    "hbpc_batch_destroy": (None, [_CTX]),
    "hbpc_batch_groups": (_I, [_CTX]),
    "hbpc_batch_ndof": (ctypes.c_longlong, [_CTX, _I]),
    "hbpc_batch_set_state": (_I, [_CTX, _I, _P, _I]),
    "hbpc_batch_get_state": (_I, [_CTX, _I, _P, _I]),
    "hbpc_batch_node_coords": (_I, [_CTX, _I, _P]),
    "hbpc_batch_eval_R1": (_I, [_CTX, _I, _P]),
    "hbpc_batch_step": (_I, [_CTX, _I]),
    "hbpc_batch_set_step_graph": (_I, [_CTX, _I]),
    "hbpc_batch_set_pc_rebuild": (_I, [_CTX, _I]),
    "hbpc_batch_get_stats": (_I, [_CTX, ctypes.POINTER(Stats)]),
    "hbpc_batch_profile_enable": (_I, [_CTX, _I]),
    "hbpc_batch_last_error": (ctypes.c_char_p, [_CTX]),
    "hbpc_autotune": (_I, [_CTX, _P]),
    "hbpc_batch_autotune": (_I, [_CTX, _P, _I]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class HBPCError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))


def _check(status, ctx=None):
    if status != OK:
        msg = _lib.hbpc_last_error(ctx)
        raise HBPCError(status, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.dtype == np.float64 and t.flags.c_contiguous
        return t.ctypes.data
    assert t.is_contiguous() and str(t.dtype) == "torch.float64"
    return t.data_ptr()


def basis(N, nodes=NODES_LOBATTO):
    p = N + 1
    xi, w, lm, lp = (np.zeros(p) for _ in range(4))
    Dh = np.zeros((p, p))
    _check(_lib.hbpc_basis(N, nodes, _ptr(xi), _ptr(w), _ptr(Dh), _ptr(lm), _ptr(lp)))
    return {"nodes": xi, "weights": w, "Dhat": Dh, "l_m": lm, "l_p": lp}


def fp64_fma_peak():
    """Measured FP64 FMA throughput of the current device, GFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(_lib.hbpc_fp64_fma_peak(ctypes.byref(v)))
    return v.value


def eval_Jv_noalloc(dim, n, lo, hi, N, dt, alpha1, alpha2, X, dX, out, law=LAW_ADVECTION,
                    flux=FLUX_GLOBAL_LF, a=(1.0, 1.0, 1.0), gamma=1.4, eps=1.0, lf_scale=1.0,
                    nodes=NODES_LOBATTO, stream=None, nu=0.0):
    """Jacobian-vector product of one stage system without a context and without
    any device allocation (hbpc_eval_Jv_noalloc; n_dof <= 262144)."""
    pad = lambda v, fill: (list(v) + [fill] * 3)[:3]
    mesh = _mesh(dim, n, lo, hi)
    phys = Physics(law, flux, (ctypes.c_double * 3)(*pad(a, 0.0)), gamma, eps, lf_scale, nu)
    _check(_lib.hbpc_eval_Jv_noalloc(ctypes.byref(mesh), N, nodes, ctypes.byref(phys), dt, alpha1,
                                     alpha2, _ptr(X), _ptr(dX), _ptr(out), stream))
    return out


class Context:
    """One HBPC-DGSEM problem on the current CUDA device.

    Arguments follow the C structs of ``include/hbpc.h``: the mesh (dim, n, lo,
    hi), the degree N and node family, the law and flux (a: advection speed;
    gamma, eps: Euler and Navier-Stokes; nu: the viscosity of a scalar law's
    BR2 term; mu, prandtl: the Navier-Stokes viscosity and Prandtl number, mu
    filling the same field as nu; eta_br2: the BR2 face factor, <= 0 for 2 dim)
    and the solver (HBPC(q, kmax), dt, Newton and GMRES tolerances, restart,
    iteration caps, preconditioner, precision).  Arrays passed to the eval_*
    and newton_solve methods are CUDA tensors in the canonical layout
    w[e][v][node]; set_state/get_state take and return numpy arrays."""

    def __init__(self, dim, n, lo, hi, N, law=LAW_ADVECTION, flux=FLUX_GLOBAL_LF,
                 a=(1.0, 1.0, 1.0), gamma=1.4, eps=1.0, lf_scale=1.0, nu=0.0, eta_br2=0.0,
                 nodes=NODES_LOBATTO, mu=None, prandtl=0.72,
                 q=4, kmax=0, dt=0.01, tol_newton_rel=1e-12, tol_newton_abs=0.0,
                 tol_gmres_rel=1e-5, gmres_restart=100, gmres_max_iter=7000,
                 newton_max_iter=50, pc=PC_NONE, precision=PREC_FP64, stream=None, t_end=0.0,
                 periodic=1):
        pad = lambda v, fill: (list(v) + [fill] * 3)[:3]
        self.mesh = _mesh(dim, n, lo, hi, periodic)
        # the Navier-Stokes law takes its dynamic viscosity mu in the nu field
        self.phys = Physics(law, flux, (ctypes.c_double * 3)(*pad(a, 0.0)), gamma, eps, lf_scale,
                            nu if mu is None else mu, eta_br2, prandtl)
        self.solver = Solver(q, kmax, dt, tol_newton_rel, tol_newton_abs, tol_gmres_rel,
                             gmres_restart, gmres_max_iter, newton_max_iter, pc, precision, t_end)
        self.N, self.dim, self.nodes = N, dim, nodes
        self._ctx = _CTX()
        _check(_lib.hbpc_create(ctypes.byref(self._ctx), ctypes.byref(self.mesh), N, nodes,
                                ctypes.byref(self.phys), ctypes.byref(self.solver), stream))
        self.ndof = _lib.hbpc_ndof(self._ctx)
        self.nv = _lib.hbpc_nvar(self._ctx)
        self.nE = 1
        for m in range(dim):
            self.nE *= n[m]
        self.shape = (self.nE, self.nv) + (N + 1,) * dim

    def close(self):
        if self._ctx:
            _lib.hbpc_destroy(self._ctx)
            self._ctx = _CTX()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        _check(st, self._ctx)

    def node_coords(self):
        nn = (self.N + 1) ** self.dim
        x = np.zeros((self.dim, self.nE * nn))
        self._c(_lib.hbpc_node_coords(self._ctx, _ptr(x)))
        return [x[m].reshape((self.nE,) + (self.N + 1,) * self.dim) for m in range(self.dim)]

    def set_state(self, w):
        on_dev = 0 if isinstance(w, np.ndarray) else 1
        if on_dev == 0:
            w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.size == self.ndof
        self._c(_lib.hbpc_set_state(self._ctx, _ptr(w), on_dev))

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(self.shape)
        on_dev = 0 if isinstance(out, np.ndarray) else 1
        self._c(_lib.hbpc_get_state(self._ctx, _ptr(out), on_dev))
        return out

    def set_state_host_ptr(self, ptr):
        """Copy the state in from host memory at address `ptr` (n_dof FP64)."""
        self._c(_lib.hbpc_set_state(self._ctx, ptr, 0))

    def get_state_host_ptr(self, ptr):
        """Copy the state out to host memory at address `ptr` (n_dof FP64)."""
        self._c(_lib.hbpc_get_state(self._ctx, ptr, 0))

    def set_time(self, t):
        self._c(_lib.hbpc_set_time(self._ctx, t))

    def step(self, n=1):
        self._c(_lib.hbpc_step(self._ctx, n))

    def advance_to(self, t_end):
        self._c(_lib.hbpc_advance_to(self._ctx, t_end))

    def run(self):
        self._c(_lib.hbpc_run(self._ctx))

    def set_wait_limit(self, seconds):
        self._c(_lib.hbpc_set_wait_limit(self._ctx, seconds))

    def set_schur(self, on=True):
        """Newton steps through the Schur-complement system of Sec. 3.2.4 (FP64)."""
        self._c(_lib.hbpc_set_schur(self._ctx, 1 if on else 0))

    def set_boundary(self, dim_index, lo, hi):
        """Boundaries of direction dim_index: lo and hi are each None (periodic;
        both or neither), "wall" (Euler slip wall), "noslip" (Navier-Stokes
        adiabatic no-slip wall) or a sequence of n_var conservative values
        (constant Dirichlet state)."""
        def kind(b):
            if b is None:
                return BC_PERIODIC, None
            if isinstance(b, str):
                if b not in ("wall", "noslip"):
                    raise ValueError(b)
                return (BC_WALL if b == "wall" else BC_NOSLIP), None
            arr = np.ascontiguousarray(np.asarray(b, dtype=np.float64).ravel())
            return BC_DIRICHLET, arr
        klo, alo = kind(lo)
        khi, ahi = kind(hi)
        p = lambda a: a.ctypes.data if a is not None else None
        self._c(_lib.hbpc_set_boundary(self._ctx, dim_index, klo, p(alo), khi, p(ahi)))

    def set_step_graph(self, on=True):
        """Every step as one CUDA graph launch (device-driven Newton and GMRES)."""
        self._c(_lib.hbpc_set_step_graph(self._ctx, 1 if on else 0))

    def set_pc_rebuild(self, every_newton_iteration=True):
        """Rebuild the block preconditioner before every Newton iteration (True)
        or once per Newton solve (False)."""
        self._c(_lib.hbpc_set_pc_rebuild(self._ctx, 1 if every_newton_iteration else 0))

    def set_corrector_batch(self, on=True):
        """Solve the s - 1 corrector stages of every sweep as one batched Newton."""
        self._c(_lib.hbpc_set_corrector_batch(self._ctx, 1 if on else 0))

    def eval_R1(self, w, out):
        self._c(_lib.hbpc_eval_R1(self._ctx, _ptr(w), _ptr(out)))
        return out

    def eval_R2(self, w, s, out):
        self._c(_lib.hbpc_eval_R2(self._ctx, _ptr(w), _ptr(s), _ptr(out)))
        return out

    def eval_G(self, b, alpha1, alpha2, X, G):
        self._c(_lib.hbpc_eval_G(self._ctx, _ptr(b), alpha1, alpha2, _ptr(X), _ptr(G)))
        return G

    def eval_Jv(self, alpha1, alpha2, X, dX, out):
        self._c(_lib.hbpc_eval_Jv(self._ctx, alpha1, alpha2, _ptr(X), _ptr(dX), _ptr(out)))
        return out

    def eval_pc(self, alpha1, alpha2, X, inp, out):
        self._c(_lib.hbpc_eval_pc(self._ctx, alpha1, alpha2, _ptr(X), _ptr(inp), _ptr(out)))
        return out

    # -- learned block preconditioner ---------------------------------------
    def set_pc(self, pc):
        self._c(_lib.hbpc_set_pc(self._ctx, pc))

    def pc_model_info(self):
        v = [ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_longlong(0)]
        self._c(_lib.hbpc_pc_model_info(self._ctx, *[ctypes.addressof(t) for t in v]))
        return {"d_in_padded": v[0].value, "hidden": v[1].value, "d_out_padded": v[2].value,
                "n_params": v[3].value}

    def pc_model_init(self, seed=0, out_scale=1e-2):
        self._c(_lib.hbpc_pc_model_init(self._ctx, seed, out_scale))

    def pc_model_get(self):
        out = np.zeros(self.pc_model_info()["n_params"], dtype=np.float32)
        self._c(_lib.hbpc_pc_model_get(self._ctx, out.ctypes.data))
        return out

    def pc_model_set(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        self._c(_lib.hbpc_pc_model_set(self._ctx, params.ctypes.data))

    def pc_loss_grad(self, F, J, c12, X=None, loss="probe"):
        # loss and gradients for host inputs; J is the element Jacobian for the
        # probe loss and the target block inverse for the inverse loss
        kind = PC_LOSS[loss]
        F, J, c12 = (np.ascontiguousarray(a, dtype=np.float32) for a in (F, J, c12))
        B = F.shape[0]
        P = 1
        xp = None
        if X is not None:
            X = np.ascontiguousarray(X, dtype=np.float32)
            P = X.shape[1]
            xp = X.ctypes.data
        out = ctypes.c_double(0.0)
        grads = np.zeros(self.pc_model_info()["n_params"], dtype=np.float32)
        self._c(_lib.hbpc_pc_loss_grad(self._ctx, kind, B, P, F.ctypes.data, J.ctypes.data, c12.ctypes.data,
                                       xp, ctypes.addressof(out), grads.ctypes.data))
        return out.value, grads

    def pc_model_forward(self, F, c12):
        """The network's blocks M~ (B x n_b x n_b) for standardised features F and (c1, c2)."""
        F = np.ascontiguousarray(F, dtype=np.float32)
        c12 = np.ascontiguousarray(c12, dtype=np.float32)
        B = F.shape[0]
        nb = self.nv * (self.N + 1) ** self.dim
        out = np.zeros((B, nb, nb), dtype=np.float32)
        self._c(_lib.hbpc_pc_model_forward(self._ctx, B, F.ctypes.data, c12.ctypes.data, out.ctypes.data))
        return out

    def pc_adam_step(self, grads, lr):
        grads = np.ascontiguousarray(grads, dtype=np.float32)
        self._c(_lib.hbpc_pc_adam_step(self._ctx, grads.ctypes.data, lr))

    def pc_collect(self, samples_per_newton, capacity):
        self._c(_lib.hbpc_pc_collect(self._ctx, samples_per_newton, capacity))

    def pc_train(self, iters, batch=256, probes=4, lr=1e-3, seed=0, loss="probe"):
        l0, l1 = ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._c(_lib.hbpc_pc_train(self._ctx, PC_LOSS[loss], iters, batch, probes, lr, seed,
                                   ctypes.addressof(l0), ctypes.addressof(l1)))
        return l0.value, l1.value

    def newton_solve(self, b, alpha1, alpha2, W0, W_out, S_out=None):
        self._c(_lib.hbpc_newton_solve(self._ctx, _ptr(b), alpha1, alpha2, _ptr(W0), _ptr(W_out),
                                       _ptr(S_out)))
        return W_out

    def stats(self):
        s = Stats()
        self._c(_lib.hbpc_get_stats(self._ctx, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def reset_stats(self):
        self._c(_lib.hbpc_reset_stats(self._ctx))

    def profile(self, enable=True):
        self._c(_lib.hbpc_profile_enable(self._ctx, 1 if enable else 0))

    def autotune(self):
        t = Tuning()
        self._c(_lib.hbpc_autotune(self._ctx, ctypes.addressof(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def profile_get(self):
        ms = np.zeros(len(PHASES))
        cnt = np.zeros(len(PHASES), dtype=np.int64)
        self._c(_lib.hbpc_profile_get(self._ctx, _ptr(ms), cnt.ctypes.data, len(PHASES)))
        return {ph: (float(ms[i]), int(cnt[i])) for i, ph in enumerate(PHASES)}


class Batch:
    """A batch of independent instances (own mesh, degree N and viscosity each)
    advanced together; see hbpc_batch_create in include/hbpc.h."""

    def __init__(self, dim, meshes, Ns, nus=None, law=LAW_BURGERS, flux=FLUX_GLOBAL_LF,
                 a=(1.0, 1.0, 1.0), gamma=1.4, eps=1.0, lf_scale=1.0, eta_br2=0.0, nodes=NODES_LOBATTO,
                 q=4, kmax=0, dt=0.01, tol_newton_rel=1e-12, tol_newton_abs=0.0, tol_gmres_rel=1e-5,
                 gmres_restart=100, gmres_max_iter=7000, newton_max_iter=50, pc=PC_NONE, precision=PREC_FP64,
                 max_per_group=0):
        """meshes: list of (n, lo, hi) per instance; max_per_group <= 0: one group per N."""
        pad = lambda v, fill: (list(v) + [fill] * 3)[:3]
        k = len(meshes)
        nus = [0.0] * k if nus is None else list(nus)
        self.M = (Mesh * k)()
        self.Ph = (Physics * k)()
        for i, (n, lo, hi) in enumerate(meshes):
            self.M[i] = _mesh(dim, n, lo, hi)
            self.Ph[i] = Physics(law, flux, (ctypes.c_double * 3)(*pad(a, 0.0)), gamma, eps, lf_scale,
                                 float(nus[i]), eta_br2, 0.72)
        self.Nv = (ctypes.c_int * k)(*Ns)
        self.solver = Solver(q, kmax, dt, tol_newton_rel, tol_newton_abs, tol_gmres_rel, gmres_restart,
                             gmres_max_iter, newton_max_iter, pc, precision)
        self.dim, self.n_inst, self.Ns = dim, k, list(Ns)
        self.nv = (dim + 2) if law in (LAW_EULER, LAW_NAVIER_STOKES) else 1
        self.meshes = [tuple(m) for m in meshes]
        self._b = _CTX()
        st = _lib.hbpc_batch_create(ctypes.byref(self._b), k, ctypes.addressof(self.M), ctypes.addressof(self.Nv),
                                    nodes, ctypes.addressof(self.Ph), ctypes.byref(self.solver), max_per_group)
        if st != OK:
            raise HBPCError(st, (_lib.hbpc_batch_last_error(None) or b"").decode())

    def _c(self, st):
        if st != OK:
            raise HBPCError(st, (_lib.hbpc_batch_last_error(self._b) or b"").decode())

    def close(self):
        if self._b:
            _lib.hbpc_batch_destroy(self._b)
            self._b = _CTX()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def groups(self):
        return _lib.hbpc_batch_groups(self._b)

    def shape(self, i):
        n = self.meshes[i][0]
        nE = int(np.prod(n[:self.dim]))
        return (nE, self.nv) + (self.Ns[i] + 1,) * self.dim

    def ndof(self, i):
        return int(_lib.hbpc_batch_ndof(self._b, i))

    def node_coords(self, i):
        shp = self.shape(i)
        out = np.zeros((self.dim, shp[0]) + shp[2:])
        self._c(_lib.hbpc_batch_node_coords(self._b, i, out.ctypes.data))
        return [out[m] for m in range(self.dim)]

    def set_state(self, i, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.size == self.ndof(i)
        self._c(_lib.hbpc_batch_set_state(self._b, i, w.ctypes.data, 0))

    def get_state(self, i):
        out = np.zeros(self.shape(i))
        self._c(_lib.hbpc_batch_get_state(self._b, i, out.ctypes.data, 0))
        return out

    def eval_R1(self, i):
        out = np.zeros(self.shape(i))
        self._c(_lib.hbpc_batch_eval_R1(self._b, i, out.ctypes.data))
        return out

    def step(self, n=1):
        self._c(_lib.hbpc_batch_step(self._b, n))

    def set_step_graph(self, on=True):
        """Every group's step as one CUDA graph launch."""
        self._c(_lib.hbpc_batch_set_step_graph(self._b, 1 if on else 0))

    def set_pc_rebuild(self, every_newton_iteration=True):
        self._c(_lib.hbpc_batch_set_pc_rebuild(self._b, 1 if every_newton_iteration else 0))

    def stats(self):
        s = Stats()
        self._c(_lib.hbpc_batch_get_stats(self._b, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def profile(self, enable=True):
        self._c(_lib.hbpc_batch_profile_enable(self._b, 1 if enable else 0))

    def autotune(self):
        k = self.groups()
        arr = (Tuning * k)()
        self._c(_lib.hbpc_batch_autotune(self._b, ctypes.addressof(arr), k))
        return [{f: getattr(arr[i], f) for f, _ in Tuning._fields_} for i in range(k)]
