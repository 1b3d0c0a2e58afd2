"""Physical fluxes F^m(w) and their directional derivatives (dF^m/dw) s for the
conservation laws of the paper.  Test infrastructure only (see
``oracle/__init__``).

Arrays carry the conserved variables on axis 0; every function is written with
plain arithmetic so that it also runs on complex arrays (complex-step tests).

  advection   F^m = a_m w                                   (Sec. 4.1.1)
  burgers     F^m = w^2 / 2 in every direction (the inviscid part; the viscous
              term nu Laplace(u) of the viscous Burgers workload is the BR2
              operator of ``dgsem.viscous``)
  euler       Eq. 21: F^m = (rho v_m, rho v_m v + p/eps^2 e_m, v_m (E + p)),
              p = (gamma - 1)(E - eps^2/2 rho |v|^2)
  navier_stokes  the Euler flux plus the viscous flux of Sec. 5 (Eq. 25):
              F^v_m = (0, tau_{k m}, sum_k tau_{m k} v_k + lambda dT/dx_m),
              tau = mu (grad v + grad v^T - 2/3 div v I), T = p / (rho R),
              R = 1 / (gamma eps^2), c_p = R gamma / (gamma - 1),
              lambda = c_p mu / Pr; its input is the gradient variable
              w_grad = (v, T) and its gradient d (Eq. 26)

Numerical-flux dissipation (Eq. 13 and its parameters in Sec. 4.1):
  global Lax-Friedrichs: lambda is a constant per variable; advection
  lambda = |a . n|, Euler lambda = diag(1/eps, 1, .., 1, 1/eps) (Sec. 4.1.2).
  Rusanov: lambda = 1/2 max(|v_n^L| + c^L, |v_n^R| + c^R), the usual local
  choice (the Euler workload asks for it); c = sqrt(gamma p / rho) / eps.
"""
import numpy as np

ADVECTION = "advection"
BURGERS = "burgers"
EULER = "euler"
NAVIER_STOKES = "navier_stokes"


class Physics:
    def __init__(self, law, dim, a=(1.0, 1.0, 1.0), gamma=1.4, eps=1.0,
                 flux="lf", lf_scale=1.0, nu=0.0, eta_br2=None, mu=0.0, prandtl=0.72):
        self.law = law
        self.dim = dim
        self.a = np.array(a[:dim], dtype=np.float64)
        self.gamma = gamma
        self.eps = eps
        self.flux = flux            # "lf" (global Lax-Friedrichs) or "rusanov"
        self.lf_scale = lf_scale    # multiplies the paper's lambda in "lf"
        self.nv = {ADVECTION: 1, BURGERS: 1, EULER: dim + 2, NAVIER_STOKES: dim + 2}[law]
        self.linear = law == ADVECTION
        # viscous term nu Laplace(w) (scalar laws only) with the BR2 lifting of
        # Sec. 6.1; eta_br2 scales the face-local liftings (the paper leaves its
        # value open; default: the number of faces of an element, 2 dim)
        if nu != 0.0 and law in (EULER, NAVIER_STOKES):
            raise ValueError("nu is the viscosity of the scalar laws; Navier-Stokes takes mu")
        if mu != 0.0 and law != NAVIER_STOKES:
            raise ValueError("mu is the dynamic viscosity of the Navier-Stokes law")
        self.nu = float(nu)
        self.eta_br2 = float(2 * dim if eta_br2 is None else eta_br2)
        # Navier-Stokes (Sec. 5): constant dynamic viscosity mu, Prandtl number,
        # gas constant R = 1/(gamma eps^2), c_p = R gamma/(gamma - 1), lambda = c_p mu/Pr
        self.mu = float(mu)
        self.prandtl = float(prandtl)
        self.R_gas = 1.0 / (gamma * eps ** 2)
        self.cp = self.R_gas * gamma / (gamma - 1.0)
        self.kappa_heat = self.cp * self.mu / self.prandtl


def _re(x):
    return np.real(x)


def cs_abs(x):
    """|x| that keeps the derivative for complex-step use (sign of the real part)."""
    return np.where(_re(x) >= 0, x, -x)


def cs_max(x, y):
    return np.where(_re(x) >= _re(y), x, y)


def euler_primitives(w, ph):
    d = ph.dim
    rho = w[0]
    v = [w[1 + k] / rho for k in range(d)]
    E = w[d + 1]
    v2 = sum(vk * vk for vk in v)
    p = (ph.gamma - 1.0) * (E - 0.5 * ph.eps ** 2 * rho * v2)
    return rho, v, E, p


def flux(w, m, ph):
    """F^m(w), direction m (0 = x)."""
    if ph.law == ADVECTION:
        return ph.a[m] * w
    if ph.law == BURGERS:
        return 0.5 * w * w
    d = ph.dim
    rho, v, E, p = euler_primitives(w, ph)
    F = np.empty_like(w)
    F[0] = w[1 + m]
    for k in range(d):
        F[1 + k] = w[1 + m] * v[k]
        if k == m:
            F[1 + k] = F[1 + k] + p / ph.eps ** 2
    F[d + 1] = v[m] * (E + p)
    return F


def flux_jvp(w, s, m, ph):
    """(dF^m/dw)(w) s, the directional derivative of the flux along s."""
    if ph.law == ADVECTION:
        return ph.a[m] * s
    if ph.law == BURGERS:
        return w * s
    d = ph.dim
    g, e2 = ph.gamma, ph.eps ** 2
    rho, v, E, p = euler_primitives(w, ph)
    srho, sE = s[0], s[d + 1]
    smom = [s[1 + k] for k in range(d)]
    # derivative of v_k = m_k / rho and of p
    dv = [(smom[k] - v[k] * srho) / rho for k in range(d)]
    v2 = sum(vk * vk for vk in v)
    vdots = sum(v[k] * smom[k] for k in range(d))
    dp = (g - 1.0) * (sE - e2 * vdots + 0.5 * e2 * v2 * srho)
    J = np.empty(s.shape, dtype=np.result_type(w, s))   # complex w: complex step in w
    J[0] = smom[m]
    for k in range(d):
        J[1 + k] = v[m] * smom[k] + v[k] * smom[m] - v[m] * v[k] * srho
        if k == m:
            J[1 + k] = J[1 + k] + dp / e2
    J[d + 1] = dv[m] * (E + p) + v[m] * (sE + dp)
    return J


def lf_lambda(ph, m):
    """Constant dissipation coefficient per variable (global LF, Eq. 13)."""
    if ph.law == ADVECTION:
        lam = np.array([abs(ph.a[m])])
    elif ph.law == BURGERS:
        lam = np.array([1.0])
    else:
        lam = np.ones(ph.nv)
        lam[0] = 1.0 / ph.eps
        lam[-1] = 1.0 / ph.eps
    return ph.lf_scale * lam


def max_speed(w, m, ph):
    """Largest |eigenvalue| of dF^m/dw at w (per point)."""
    if ph.law == ADVECTION:
        return np.full(w.shape[1:], abs(ph.a[m]))
    if ph.law == BURGERS:
        return cs_abs(w[0])
    rho, v, E, p = euler_primitives(w, ph)
    c = np.sqrt(ph.gamma * p / rho) / ph.eps
    return cs_abs(v[m]) + c


def dissipation(wL, wR, m, ph):
    """The coefficient kappa multiplying (w^L - w^R) in the numerical flux;
    broadcastable against a state array with variables on axis 0."""
    if ph.flux == "lf":
        lam = lf_lambda(ph, m)
        return lam.reshape((-1,) + (1,) * (wL.ndim - 1))
    if ph.flux == "rusanov":
        return 0.5 * cs_max(max_speed(wL, m, ph), max_speed(wR, m, ph))[None]
    raise ValueError(ph.flux)


# -- boundary exteriors (non-periodic directions) ----------------------------

def exterior_state(w_own, spec, m, ph):
    """The state the numerical flux sees outside a boundary face of direction
    m, from the element's own trace w_own (variables on axis 0):
      ("dirichlet", state): the given constant state;
      ("wall",): the Euler slip wall, the own state with its momentum along m
                 reversed (zero normal velocity at the face);
      ("noslip",): the Navier-Stokes no-slip adiabatic wall, the own state
                 with its whole momentum reversed (zero velocity at the face)."""
    if spec[0] == "dirichlet":
        st = np.asarray(spec[1], dtype=np.float64).reshape((ph.nv,) + (1,) * (w_own.ndim - 1))
        return np.broadcast_to(st, w_own.shape).astype(np.result_type(w_own, st))
    if spec[0] == "wall":
        if ph.law != EULER:
            raise ValueError("a slip wall needs the Euler equations")
        out = np.array(w_own, copy=True)
        out[1 + m] = -out[1 + m]
        return out
    if spec[0] == "noslip":
        if ph.law != NAVIER_STOKES:
            raise ValueError("a no-slip wall needs the Navier-Stokes equations")
        out = np.array(w_own, copy=True)
        for k in range(ph.dim):
            out[1 + k] = -out[1 + k]
        return out
    raise ValueError(spec)


def exterior_direction(s_own, spec, m, ph):
    """The direction sigma outside a boundary face: the time derivative of the
    exterior state, so zero for constant Dirichlet data and the mirrored own
    sigma at a wall (the exterior state is linear in the own state)."""
    if spec[0] == "dirichlet":
        return np.zeros_like(s_own)
    return exterior_state(s_own, spec, m, ph)


# -- Navier-Stokes viscous part (Sec. 5) -----------------------------------

def ns_grad_vars(w, ph):
    """w_grad = (v_1, .., v_d, T) of Eq. 26, T = p / (rho R)."""
    rho, v, E, p = euler_primitives(w, ph)
    return np.stack(v + [p / (rho * ph.R_gas)])


def ns_grad_vars_jvp(w, s, ph):
    """(d w_grad / dw) s: the velocity and temperature parts of the direction s
    (the matrix of Eq. 31 applied to sigma)."""
    d = ph.dim
    g, e2 = ph.gamma, ph.eps ** 2
    rho, v, E, p = euler_primitives(w, ph)
    srho, sE = s[0], s[d + 1]
    smom = [s[1 + k] for k in range(d)]
    dv = [(smom[k] - v[k] * srho) / rho for k in range(d)]
    v2 = sum(vk * vk for vk in v)
    vdots = sum(v[k] * smom[k] for k in range(d))
    dp = (g - 1.0) * (sE - e2 * vdots + 0.5 * e2 * v2 * srho)
    dT = (dp / rho - p * srho / (rho * rho)) / ph.R_gas
    return np.stack(dv + [dT])


def _tau(dg, i, j, ph):
    """tau_ij = mu (dv_j/dx_i + dv_i/dx_j - 2/3 delta_ij div v); dg[k][c] is the
    derivative of gradient variable c along x_k."""
    t = dg[i][j] + dg[j][i]
    if i == j:
        t = t - (2.0 / 3.0) * sum(dg[k][k] for k in range(ph.dim))
    return ph.mu * t


def ns_viscous_flux(g, dg, m, ph):
    """F^v along x_m (Eq. 25) from the gradient variables g = (v, T) and their
    gradient dg (dg[k][c] = d g_c / d x_k):
    (0, tau_{k m} for k < d, sum_k tau_{m k} v_k + lambda dT/dx_m)."""
    d = ph.dim
    zero = 0.0 * g[0]
    rows = [zero]
    for k in range(d):
        rows.append(_tau(dg, k, m, ph))
    energy = ph.kappa_heat * dg[m][d]
    for k in range(d):
        energy = energy + _tau(dg, m, k, ph) * g[k]
    rows.append(energy)
    return np.stack(rows)


def ns_viscous_flux_jvp(g, dg, gs, dgs, m, ph):
    """The linearisation of ns_viscous_flux in the direction (gs, dgs) of
    (g, d): tau is linear in d and independent of w, so (Eq. 32)
    (0, tau(dgs)_{k m}, sum_k [tau(dgs)_{m k} v_k + tau(dg)_{m k} gs_k] + lambda dgs[m][T])."""
    d = ph.dim
    zero = 0.0 * g[0]
    rows = [zero]
    for k in range(d):
        rows.append(_tau(dgs, k, m, ph))
    energy = ph.kappa_heat * dgs[m][d]
    for k in range(d):
        energy = energy + _tau(dgs, m, k, ph) * g[k] + _tau(dg, m, k, ph) * gs[k]
    rows.append(energy)
    return np.stack(rows)
