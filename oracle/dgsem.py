"""DGSEM operators R^(1) (Eq. 12) and R^(2) (Eq. 16) on periodic, uniform
Cartesian meshes in 1, 2 or 3 dimensions.  Test infrastructure only (see
``oracle/__init__``).

State layout (canonical, shared with the library's C-ABI):
    w[e][v][k][j][i]   (i = x node index fastest; d = 1, 2, 3 keeps the last d
                        node axes), e = ex + nx * (ey + ny * ez).

On a Cartesian element of size h_m the transformation of Sec. 3.1.1 reduces to
J_geo = prod h_m / 2, transformed flux (prod_{n != m} h_n/2) F^m and surface
element of the same size, so Eq. 12 becomes, for every direction m,

    R1 += -(2 / h_m) [ sum_l Dhat[i, l] F^m_l  +  f*_{+m} lhat_i(+1)
                                               +  f*_{-m} lhat_i(-1) ]

along the node index of direction m, where f*_{+-m} is the numerical flux of
Eq. 13 with the outward normal of that face and w^L the element's own trace.
Traces are the solution polynomial evaluated at the edge (Sec. 3.1.1).

R^(2)(w, sigma) is the same operator with F^m(w) replaced by (dF^m/dw) sigma and
the face flux f~* of Sec. 3.1.2, which uses the traces of w and sigma and the
same dissipation coefficient (evaluated at w, not differentiated).

Scalar laws may carry a viscous term nu Laplace(w), discretised with the BR2
lifting of Sec. 5.1.1 (``viscous``).  Its flux F^v = nu d does not depend on w,
so it adds nu L_h(w) to R^(1) and, by Eq. 31-33 with dF^v/dw = 0 and
eta = d_t, nu L_h(sigma) to R^(2).  The Navier-Stokes law adds the viscous
flux of Eq. 25 with the same lifting applied to w_grad = (v, T)
(``viscous_ns``).
"""
import numpy as np

from . import laws
from .basis import Basis, LOBATTO


class Mesh:
    """Uniform Cartesian mesh.  bc: None (periodic in every direction) or one
    entry per direction, None (periodic) or a pair (lower, upper) of boundary
    specifications ("dirichlet", state) (a constant exterior state of n_var
    values) or ("wall",) (slip wall of the Euler equations)."""

    def __init__(self, dim, n, lo, hi, bc=None):
        self.dim = dim
        self.n = tuple(int(x) for x in n[:dim])
        self.lo = np.array(lo[:dim], dtype=np.float64)
        self.hi = np.array(hi[:dim], dtype=np.float64)
        self.h = (self.hi - self.lo) / np.array(self.n)
        self.nE = int(np.prod(self.n))
        self.bc = [None] * dim if bc is None else list(bc)
        assert len(self.bc) == dim
        self.periodic = all(b is None for b in self.bc)


class Disc:
    """A discretisation: mesh + basis + physics."""

    def __init__(self, mesh, N, physics, family=LOBATTO):
        self.mesh = mesh
        self.basis = Basis(N, family)
        self.ph = physics
        self.d = mesh.dim
        self.p = N + 1
        self.nv = physics.nv
        self.shape = (mesh.nE, self.nv) + (self.p,) * self.d
        self.ndof = int(np.prod(self.shape))

    # -- layout ---------------------------------------------------------
    def to_grid(self, w):
        """canonical (nE, nv, P..) -> (nv, n_{d-1}, .., n_0, P_{d-1}, .., P_0)."""
        d = self.d
        g = w.reshape(tuple(reversed(self.mesh.n)) + (self.nv,) + (self.p,) * d)
        return np.moveaxis(g, d, 0)

    def from_grid(self, g):
        d = self.d
        w = np.moveaxis(g, 0, d)
        return w.reshape(self.shape)

    def elem_axis(self, m):
        return 1 + (self.d - 1 - m)

    def node_axis(self, m):
        return 1 + self.d + (self.d - 1 - m)

    def node_coords(self):
        """Physical coordinates of every node, list of d arrays in canonical
        shape (nE, P..) (variable axis dropped)."""
        d, mesh, xi = self.d, self.mesh, self.basis.nodes
        coords = []
        for m in range(d):
            shp = [1] * (2 * d)
            e = np.arange(mesh.n[m], dtype=np.float64)
            shp_e = list(shp)
            shp_e[d - 1 - m] = mesh.n[m]
            shp_n = list(shp)
            shp_n[d + d - 1 - m] = self.p
            x = (mesh.lo[m] + mesh.h[m] * e.reshape(shp_e)
                 + 0.5 * mesh.h[m] * (xi.reshape(shp_n) + 1.0))
            full = np.broadcast_to(x, tuple(reversed(mesh.n)) + (self.p,) * d)
            coords.append(np.ascontiguousarray(full).reshape((mesh.nE,) + (self.p,) * d))
        return coords

    # -- helpers ----------------------------------------------------------
    @staticmethod
    def _apply(M, A, axis):
        """(M A) along `axis`: out[..i..] = sum_l M[i, l] A[..l..]."""
        return np.moveaxis(np.tensordot(M, A, axes=([1], [axis])), 0, axis)

    @staticmethod
    def _trace(vec, A, axis):
        """Evaluate the polynomial along `axis` with the weights `vec` (removes axis)."""
        return np.tensordot(A, vec, axes=([axis], [0]))

    def _lift(self, f, lhat, axis):
        shp = [1] * (2 * self.d + 1)
        shp[axis] = self.p
        return np.expand_dims(f, axis) * lhat.reshape(shp)


def _end(ndim, axis, last):
    """Index of the first (last = False) or last element along `axis`, axis kept."""
    idx = [slice(None)] * ndim
    idx[axis] = slice(-1, None) if last else slice(0, 1)
    return tuple(idx)


def _neighbour_traces(disc, own_p, own_m, m, ea, exterior, nb=None):
    """The traces the element's faces see across them along direction m:
    L at its - face (the + trace of element e-1) and R at its + face (the -
    trace of element e+1).  nb (optional) maps the rolled neighbour values
    (real parts, zeros).  On a bounded direction the first element's L and
    the last element's R are the exterior values exterior(own trace, spec)."""
    R = np.roll(own_m, -1, axis=ea)
    L = np.roll(own_p, 1, axis=ea)
    if nb is not None:
        R, L = nb(R), nb(L)
    bc = disc.mesh.bc[m]
    if bc is not None:
        lo, hi = bc
        dt = np.result_type(R, own_p)
        R, L = R.astype(dt, copy=True), L.astype(dt, copy=True)
        e_hi, e_lo = _end(R.ndim, ea, True), _end(L.ndim, ea, False)
        R[e_hi] = exterior(own_p[e_hi], hi)
        L[e_lo] = exterior(own_m[e_lo], lo)
    return L, R


def operator(disc, w, sigma=None, mode="R1", frozen_neighbor=False, frozen_neighbor_state=False):
    """R^(1)(w) if mode == "R1"; R^(2)(w, sigma) if mode == "R2".

    frozen_neighbor (R2 only): the neighbours' sigma traces are taken as zero,
    which gives the element-local linearisation used by the block
    preconditioners of Sec. 3.2.3 (neighbour dependencies neglected).

    frozen_neighbor_state (R2 only, inviscid and scalar viscous laws): for a
    complex state w, the neighbours' state traces enter with their real parts
    and the dissipation coefficient kappa is that of the real traces, so that
    Im R2(W + i h e_k, sigma) / h is the derivative of R2 with respect to the
    element's own node k at fixed sigma and fixed neighbour states: the
    element block of dR2/dW, where the physical flux Jacobians of the
    assembly are replaced by the physical flux Hessians (Sec. 3.2.2); the
    dissipation coefficient is not differentiated."""
    if frozen_neighbor and frozen_neighbor_state:
        raise ValueError("frozen_neighbor and frozen_neighbor_state exclude each other")
    if frozen_neighbor_state and (mode != "R2" or disc.ph.law == laws.NAVIER_STOKES):
        raise ValueError("frozen_neighbor_state: R2 of an inviscid or scalar viscous law only")
    ph, b = disc.ph, disc.basis
    if not disc.mesh.periodic and ph.nu != 0.0:
        raise ValueError("boundary conditions: not for the scalar viscous term")
    W = disc.to_grid(w)
    S = disc.to_grid(sigma) if sigma is not None else None
    out = np.zeros(W.shape, dtype=np.result_type(W, S) if S is not None else W.dtype)
    for m in range(disc.d):
        ea, na = disc.elem_axis(m), disc.node_axis(m)
        # nodal flux and volume term
        if mode == "R1":
            F = laws.flux(W, m, ph)
        else:
            F = laws.flux_jvp(W, S, m, ph)
        vol = Disc._apply(b.Dhat, F, na)
        # traces: own + face (right trace) and own - face (left trace)
        wp = Disc._trace(b.l_p, W, na)
        wm = Disc._trace(b.l_m, W, na)
        ext_w = lambda own, spec: laws.exterior_state(own, spec, m, ph)
        # neighbours' traces: wL at the - face (e-1's + trace), wR at the +
        # face (e+1's - trace); real parts when the neighbours are frozen
        wL, wR = _neighbour_traces(disc, wp, wm, m, ea, ext_w,
                                   np.real if frozen_neighbor_state else None)
        if frozen_neighbor_state:
            kp = laws.dissipation(np.real(wp), np.real(wR), m, ph)
            km = laws.dissipation(np.real(wL), np.real(wm), m, ph)
        else:
            kp = laws.dissipation(wp, wR, m, ph)
            km = laws.dissipation(wL, wm, m, ph)
        if mode == "R1":
            # + face: f*(own, e+1); - face: -f*(e-1, own) (outward normal -e_m)
            fplus = 0.5 * (laws.flux(wp, m, ph) + laws.flux(wR, m, ph)) + kp * (wp - wR)
            fminus = -(0.5 * (laws.flux(wL, m, ph) + laws.flux(wm, m, ph)) + km * (wL - wm))
        else:
            sp = Disc._trace(b.l_p, S, na)
            sm = Disc._trace(b.l_m, S, na)
            ext_s = lambda own, spec: laws.exterior_direction(own, spec, m, ph)
            # frozen_neighbor: the neighbours' sigma traces are zero (an
            # exterior value stays: it is the element's own)
            sL, sR = _neighbour_traces(disc, sp, sm, m, ea, ext_s,
                                       np.zeros_like if frozen_neighbor else None)
            fplus = (0.5 * (laws.flux_jvp(wp, sp, m, ph) + laws.flux_jvp(wR, sR, m, ph))
                     + kp * (sp - sR))
            fminus = -(0.5 * (laws.flux_jvp(wL, sL, m, ph) + laws.flux_jvp(wm, sm, m, ph))
                       + km * (sL - sm))
        surf = disc._lift(fplus, b.lhat_p, na) + disc._lift(fminus, b.lhat_m, na)
        out = out - (2.0 / disc.mesh.h[m]) * (vol + surf)
    res = disc.from_grid(out)
    if ph.nu != 0.0:
        res = res + viscous(disc, w if mode == "R1" else sigma, frozen_neighbor and mode == "R2")
    if ph.law == laws.NAVIER_STOKES and ph.mu != 0.0:
        res = res + viscous_ns(disc, w, sigma if mode == "R2" else None, frozen_neighbor and mode == "R2")
    return res


def br2_traces(disc, U, m, frozen_neighbor=False):
    """Face quantities of the BR2 lifting along direction m (Sec. 5.1.1) for a
    scalar grid array U: the common value u* of Eq. 30 at the element's + and
    - faces and the face gradients d^L, d^R of the face-local liftings.

    The face-local lifting of a face f (strong form; equal to the weak form on
    the collocated nodes) keeps only f's surface term, scaled by eta:
        d_f = (2/h) D u + eta r_f,   (r_f, phi) = <(u* - u) n, phi>_f,
    evaluated at f.  On the element's + face (n = +e_m) this gives
    d = (2/h)[u'(+1) + eta c_p (u* - u(+1))], on its - face (n = -e_m)
    d = (2/h)[u'(-1) + eta c_m (u(-1) - u*)], with c_pm = sum_i l_i(pm1)^2 / omega_i.
    frozen_neighbor: the neighbours' values are taken as zero.
    Returns (ustar_p, ustar_m, fp_grad, fm_grad): u* at the + and - faces and the
    averages 1/2 (d^L + d^R) at the + and - faces (gradient along +e_m)."""
    ph, b = disc.ph, disc.basis
    ea, na = disc.elem_axis(m), disc.node_axis(m)
    H = 2.0 / disc.mesh.h[m]
    eta = ph.eta_br2
    c_p = float(np.sum(b.l_p * b.lhat_p))
    c_m = float(np.sum(b.l_m * b.lhat_m))
    dl_p = b.l_p @ b.D      # l_j'(+1): derivative of the interpolant at +1
    dl_m = b.l_m @ b.D
    up = Disc._trace(b.l_p, U, na)
    um = Disc._trace(b.l_m, U, na)
    gp = H * Disc._trace(dl_p, U, na)
    gm = H * Disc._trace(dl_m, U, na)
    if not frozen_neighbor:
        uR = np.roll(um, -1, axis=ea)          # right neighbour's - trace
        gR = np.roll(gm, -1, axis=ea)
        ustar_p = 0.5 * (up + uR)
        dL = gp + H * eta * c_p * (ustar_p - up)
        dR = gR + H * eta * c_m * (uR - ustar_p)
        fp_grad = 0.5 * (dL + dR)
        ustar_m = np.roll(ustar_p, 1, axis=ea)
        fm_grad = np.roll(fp_grad, 1, axis=ea)
    else:
        ustar_p = 0.5 * up
        fp_grad = 0.5 * ((gp + H * eta * c_p * (ustar_p - up)) + H * eta * c_m * (0.0 - ustar_p))
        ustar_m = 0.5 * um
        fm_grad = 0.5 * (H * eta * c_p * (ustar_m - 0.0) + (gm + H * eta * c_m * (um - ustar_m)))
    return ustar_p, ustar_m, fp_grad, fm_grad


def br2_gradient(disc, u, m, frozen_neighbor=False):
    """The lifted gradient component d^m of Eq. 29 (weak form, collocated):
    d_i = (2/h_m) [ sum_j Dhat[i, j] u_j + lhat_i(+1) u*_+ - lhat_i(-1) u*_- ]."""
    b = disc.basis
    U = disc.to_grid(u)
    na = disc.node_axis(m)
    ustar_p, ustar_m, _, _ = br2_traces(disc, U, m, frozen_neighbor)
    H = 2.0 / disc.mesh.h[m]
    d = H * (Disc._apply(b.Dhat, U, na) + disc._lift(ustar_p, b.lhat_p, na)
             - disc._lift(ustar_m, b.lhat_m, na))
    return disc.from_grid(d)


def viscous(disc, u, frozen_neighbor=False):
    """nu L_h(u): the viscous part of the weak form of Sec. 5.1.1 for the flux
    F^v = nu d (scalar law, constant viscosity), with the central viscous face
    flux of Eq. 30:
        out_i = sum_m (2/h_m) [ sum_j Dhat[i, j] nu d^m_j
                                + lhat_i(+1) F^v*_+ - lhat_i(-1) F^v*_- ],
    F^v*_pm = nu 1/2 (d^L + d^R) at the element's + and - faces (along +e_m).
    frozen_neighbor: neighbours' values zero (the element-diagonal block)."""
    ph, b = disc.ph, disc.basis
    U = disc.to_grid(u)
    out = np.zeros(U.shape, dtype=U.dtype)
    for m in range(disc.d):
        na = disc.node_axis(m)
        H = 2.0 / disc.mesh.h[m]
        _, _, fp_grad, fm_grad = br2_traces(disc, U, m, frozen_neighbor)
        d = disc.to_grid(br2_gradient(disc, u, m, frozen_neighbor))
        out = out + H * (Disc._apply(b.Dhat, ph.nu * d, na)
                         + disc._lift(ph.nu * fp_grad, b.lhat_p, na)
                         - disc._lift(ph.nu * fm_grad, b.lhat_m, na))
    return disc.from_grid(out)


def ns_channel_ghost(disc, spec, own_val, own_grads, m, linear):
    """The values and the broken gradient of the gradient channels (v, T) of
    Eq. 26 outside a boundary face of direction m, from the element's own
    traces there (own_grads[k]: the own d/dx_k traced on the face).  The
    exterior gradient is the own one, except that an adiabatic wall reverses
    the normal derivative of T:
      ("noslip",): adiabatic no-slip wall: the velocity reversed (u* = 0), T
          kept; the velocity gradient kept, so that the central viscous flux
          takes the wall shear stress of the own side and does no work at the
          wall, and dT/dn reversed, so that no heat crosses it;
      ("dirichlet", state): the channels of the given state (zero for the
          linearised channels, linear=True), the own gradient."""
    d = disc.d
    shp = (d + 1,) + (1,) * (own_val.ndim - 1)
    if spec[0] == "noslip":
        s_val = np.array([-1.0] * d + [1.0]).reshape(shp)
        s_nrm = np.array([1.0] * d + [-1.0]).reshape(shp)
        val = s_val * own_val
        grads = [s_nrm * gk if k == m else gk for k, gk in enumerate(own_grads)]
        return val, grads
    if spec[0] == "dirichlet":
        if linear:
            val = np.zeros_like(own_val)
        else:
            st = np.asarray(spec[1], dtype=np.float64).reshape((disc.nv,) + (1,) * (own_val.ndim - 1))
            val = np.broadcast_to(laws.ns_grad_vars(st, disc.ph), own_val.shape).astype(own_val.dtype)
        return val, list(own_grads)
    raise ValueError(spec)


def br2_faces(disc, U, m, frozen_neighbor=False, linear=False):
    """BR2 face quantities of a grid array of channels U (channels on axis 0)
    along direction m, for systems (Sec. 5.1.1): the broken gradient of every
    channel (all d components, tangential ones included, as the viscous flux
    of a system needs them) traced on the element's + and - faces, the
    neighbours' values across those faces, the common value u* of Eq. 30 and
    the face-local lifting that adds eta c_pm (2/h_m)(u* - u_own) to the normal
    component (the same lifting as ``br2_traces``).
    frozen_neighbor: the neighbours' channel values are taken as zero.
    On a bounded direction the first and last elements see the exterior
    channels of ``ns_channel_ghost`` (linear: U holds linearised channels).
    Returns dict with, for the + face ('p') and the - face ('m') of every
    element, the left and right traces gL, gR (channels) and gradients dL, dR
    (lists over the direction k of channel arrays) and u*."""
    b = disc.basis
    ph = disc.ph
    ea, na = disc.elem_axis(m), disc.node_axis(m)
    eta = ph.eta_br2
    H = 2.0 / disc.mesh.h[m]
    c_p = float(np.sum(b.l_p * b.lhat_p))
    c_m = float(np.sum(b.l_m * b.lhat_m))
    # broken gradient at the nodes, then traced on the two faces of direction m
    DU = [(2.0 / disc.mesh.h[k]) * Disc._apply(b.D, U, disc.node_axis(k)) for k in range(disc.d)]
    up = Disc._trace(b.l_p, U, na)
    um = Disc._trace(b.l_m, U, na)
    gp = [Disc._trace(b.l_p, x, na) for x in DU]
    gm = [Disc._trace(b.l_m, x, na) for x in DU]
    if frozen_neighbor:
        nb_m, nb_gm = 0.0 * um, [0.0 * x for x in gm]    # right neighbour's - face
        nb_p, nb_gp = 0.0 * up, [0.0 * x for x in gp]    # left neighbour's + face
    else:
        nb_m, nb_gm = np.roll(um, -1, axis=ea), [np.roll(x, -1, axis=ea) for x in gm]
        nb_p, nb_gp = np.roll(up, 1, axis=ea), [np.roll(x, 1, axis=ea) for x in gp]
    bc = disc.mesh.bc[m]
    if bc is not None:
        dt = np.result_type(up, nb_m)
        nb_m, nb_p = nb_m.astype(dt, copy=True), nb_p.astype(dt, copy=True)
        nb_gm = [x.astype(dt, copy=True) for x in nb_gm]
        nb_gp = [x.astype(dt, copy=True) for x in nb_gp]
        e_hi, e_lo = _end(up.ndim, ea, True), _end(up.ndim, ea, False)
        v, gs = ns_channel_ghost(disc, bc[1], up[e_hi], [x[e_hi] for x in gp], m, linear)
        nb_m[e_hi] = v
        for k in range(disc.d):
            nb_gm[k][e_hi] = gs[k]
        v, gs = ns_channel_ghost(disc, bc[0], um[e_lo], [x[e_lo] for x in gm], m, linear)
        nb_p[e_lo] = v
        for k in range(disc.d):
            nb_gp[k][e_lo] = gs[k]
    # + face: left = own, right = neighbour
    us_p = 0.5 * (up + nb_m)
    dL_p = list(gp)
    dL_p[m] = gp[m] + H * eta * c_p * (us_p - up)
    dR_p = list(nb_gm)
    dR_p[m] = nb_gm[m] + H * eta * c_m * (nb_m - us_p)
    # - face: left = neighbour, right = own
    us_m = 0.5 * (nb_p + um)
    dL_m = list(nb_gp)
    dL_m[m] = nb_gp[m] + H * eta * c_p * (us_m - nb_p)
    dR_m = list(gm)
    dR_m[m] = gm[m] + H * eta * c_m * (um - us_m)
    return {"p": dict(gL=up, gR=nb_m, dL=dL_p, dR=dR_p, us=us_p),
            "m": dict(gL=nb_p, gR=um, dL=dL_m, dR=dR_m, us=us_m)}


def br2_lifted_gradient(disc, U, faces):
    """The lifted gradient d (Eq. 29, weak form on the collocated nodes) of every
    channel of U, all directions: d^k = (2/h_k)[Dhat U + lhat(+1) u*_+ - lhat(-1) u*_-]
    along the node axis of k, with u* of ``br2_faces`` (faces[k])."""
    b = disc.basis
    out = []
    for k in range(disc.d):
        nk = disc.node_axis(k)
        Hk = 2.0 / disc.mesh.h[k]
        out.append(Hk * (Disc._apply(b.Dhat, U, nk) + disc._lift(faces[k]["p"]["us"], b.lhat_p, nk)
                         - disc._lift(faces[k]["m"]["us"], b.lhat_m, nk)))
    return out


def viscous_ns(disc, w, sigma=None, frozen_neighbor=False):
    """The viscous part of the Navier-Stokes operators (Sec. 5.1).

    R^(1) (sigma None), Eq. 28-30: the gradient variables g = w_grad(w) of
    Eq. 26 at the nodes, their lifted gradient d (Eq. 29), and
        out_i = sum_m (2/h_m)[ Dhat F^v_m(g, d) + lhat_i(+1) F^v*_+ - lhat_i(-1) F^v*_- ]
    with the central viscous face flux of Eq. 30,
        F^v*_pm = 1/2 (F^v_m(g^L, d^L) + F^v_m(g^R, d^R)),
    where g^L,R are the traces of the nodal g and d^L,R the face-local BR2
    gradients (``br2_faces``).
    R^(2) (sigma given), Eq. 32-33: the same structure with the linearised flux
    (dF^v/dw) sigma + (dF^v/dd) eta, where eta is the lifting (Eq. 33) of
    gs = (dw_grad/dw) sigma, built exactly like d from g.  frozen_neighbor
    zeroes the neighbours' gs (their sigma), not their g."""
    ph, b = disc.ph, disc.basis
    W = disc.to_grid(w)
    g = laws.ns_grad_vars(W, ph)
    fg = [br2_faces(disc, g, m) for m in range(disc.d)]
    dg = br2_lifted_gradient(disc, g, fg)
    if sigma is not None:
        S = disc.to_grid(sigma)
        gs = laws.ns_grad_vars_jvp(W, S, ph)
        fs = [br2_faces(disc, gs, m, frozen_neighbor, linear=True) for m in range(disc.d)]
        ds = br2_lifted_gradient(disc, gs, fs)
    out = np.zeros(W.shape, dtype=np.result_type(W, sigma) if sigma is not None else W.dtype)
    for m in range(disc.d):
        na = disc.node_axis(m)
        H = 2.0 / disc.mesh.h[m]
        fp, fm = fg[m]["p"], fg[m]["m"]
        if sigma is None:
            Fv = laws.ns_viscous_flux(g, dg, m, ph)
            fstar_p = 0.5 * (laws.ns_viscous_flux(fp["gL"], fp["dL"], m, ph)
                             + laws.ns_viscous_flux(fp["gR"], fp["dR"], m, ph))
            fstar_m = 0.5 * (laws.ns_viscous_flux(fm["gL"], fm["dL"], m, ph)
                             + laws.ns_viscous_flux(fm["gR"], fm["dR"], m, ph))
        else:
            sp, sm = fs[m]["p"], fs[m]["m"]
            Fv = laws.ns_viscous_flux_jvp(g, dg, gs, ds, m, ph)
            fstar_p = 0.5 * (laws.ns_viscous_flux_jvp(fp["gL"], fp["dL"], sp["gL"], sp["dL"], m, ph)
                             + laws.ns_viscous_flux_jvp(fp["gR"], fp["dR"], sp["gR"], sp["dR"], m, ph))
            fstar_m = 0.5 * (laws.ns_viscous_flux_jvp(fm["gL"], fm["dL"], sm["gL"], sm["dL"], m, ph)
                             + laws.ns_viscous_flux_jvp(fm["gR"], fm["dR"], sm["gR"], sm["dR"], m, ph))
        out = out + H * (Disc._apply(b.Dhat, Fv, na) + disc._lift(fstar_p, b.lhat_p, na)
                         - disc._lift(fstar_m, b.lhat_m, na))
    return disc.from_grid(out)


def R1(disc, w):
    """R^(1)_h(w), Eq. 12 (with Eq. 13 at the faces)."""
    return operator(disc, w, mode="R1")


def R2(disc, w, sigma):
    """R^(2)_h(w, sigma), Eq. 16."""
    return operator(disc, w, sigma, mode="R2")


def cell_integral(disc, w):
    """Integral of each variable over the domain with the collocated quadrature:
    sum_e sum_nodes (prod_m omega * h_m / 2) w.  Shape (nv,)."""
    wq = disc.basis.weights
    W = w.reshape((disc.mesh.nE, disc.nv) + (disc.p,) * disc.d)
    tot = W
    for _ in range(disc.d):
        tot = np.tensordot(tot, wq, axes=([tot.ndim - 1], [0]))
    jac = np.prod(disc.mesh.h / 2.0)
    return jac * tot.sum(axis=0)
