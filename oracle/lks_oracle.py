"""Plain FP64 CPU oracle of the lattice kinetic scheme with grid-separated moving rigid bodies.

TEST INFRASTRUCTURE ONLY.  This module is the independent checker of the CUDA path.  Only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code, table or helper with the CUDA library and never imports the product package.

Every function follows one passage of "4D Topology optimization of moving rigid bodies in fluid flows"
(Tanabe, Yaji, Ushijima), cited by section and equation label.  Arrays are indexed by spatial axis in
math order: a scalar field has shape ``(nx, ny)`` or ``(nx, ny, nz)``; a vector field has a leading axis of
length d.  Lattice units are used throughout (grid spacing and time step equal 1).  All indexing wraps
periodically on every axis (wall planes are imposed on top, see ``lks_step``).

The code is written to work unchanged on complex128 arrays, so that the tests can take exact
directional derivatives by the complex-step method (the only real-valued decisions are the integer tap
positions of the mapping kernel, taken from the real part).

Pinned by the tests in ``tests/test_oracle_*.py``: lattice isotropy, the equilibrium's zeroth, first and second
moments against their closed forms (the second moment's u_a u_b fixes the scale of the quadratic terms), the
exact shear-wave decay factor,
uniform Brinkman relaxation, Couette / Brinkman-channel steady states against a direct linear solve,
mass and momentum conservation, mapping partition of unity / shift invariance / brute force / transpose,
filter invariants and transposes, the adjoint against complex-step JVPs and central finite
differences, the objective J1 against numpy's sample mean and variance, and the rotated-body mapping (quarter
turns against ``numpy.rot90``, kept totals, the first moment turned by e^{i theta}, the rigid rotation's angular
moment, complex-step derivatives, the adjoint with angle knots by complex step and central differences), and the
oar objective J2 (uniform flow, fluid in rigid motion with the body, spinning and translating bodies in still
fluid; its adjoint by complex step and central differences).  The paper's own objective values (Sec. 4.1 table) depend on figure-only geometry:
parity unpinned for that full-problem value only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------------------------
# Lattice velocity sets (Sec. 2.2, Fig. "Velocity sets").  The paper shows the weights only in a
# figure; these are the standard D2Q9 / D3Q15 weights, pinned by the isotropy identities in the tests.
# ---------------------------------------------------------------------------------------------


def lattice(name: str):
    """Return (c, w): integer velocities c[Q, d] and weights w[Q] of D2Q9 or D3Q15 (Sec. 2.2)."""
    if name == "D2Q9":
        c = [(0, 0)]
        w = [4.0 / 9.0]
        for v in [(1, 0), (0, 1), (-1, 0), (0, -1)]:
            c.append(v)
            w.append(1.0 / 9.0)
        for v in [(1, 1), (-1, 1), (-1, -1), (1, -1)]:
            c.append(v)
            w.append(1.0 / 36.0)
    elif name == "D3Q15":
        c = [(0, 0, 0)]
        w = [2.0 / 9.0]
        for a in range(3):
            for sgn in (1, -1):
                v = [0, 0, 0]
                v[a] = sgn
                c.append(tuple(v))
                w.append(1.0 / 9.0)
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    c.append((sx, sy, sz))
                    w.append(1.0 / 72.0)
    else:
        raise ValueError(f"unknown lattice {name!r}")
    return np.array(c, dtype=np.int64), np.array(w, dtype=np.float64)


def viscosity_A(nu: float) -> float:
    """A = 3/4 - (9/2) nu / dx with dx = 1 (Sec. 2.2, Eq. for A)."""
    return 0.75 - 4.5 * nu


# ---------------------------------------------------------------------------------------------
# Problem description.  Plain data; built by the tests from the workload description.
# ---------------------------------------------------------------------------------------------


@dataclass
class Problem:
    lattice: str                      # "D2Q9" or "D3Q15"
    shape: tuple                      # analysis grid (nx, ny[, nz])
    periodic: tuple                   # per axis: True = periodic, False = wall planes at 0 and n-1
    nu: float                         # lattice kinematic viscosity
    design: tuple                     # inner design grid (ndx, ndy[, ndz])
    margin: int = 2                   # fluid margin around the design grid (Sec. 2.3), gamma = 0 there
    kappa_max: float = 1.0            # kappa_max^ref of Eq. kappa_ref
    q: float = 0.1                    # convexity parameter q of Eq. kappa_ref
    kernel: str = "linear"            # "linear" (hat, the configs) or "cosine" (Sec. 2.3 w(r))
    base_center: tuple | None = None  # analysis coordinates of the design centre at zero offset
    Nt: int = 10                      # number of time steps
    K: int = 2                        # number of motion knots
    R_t: float = 1.0                  # temporal filter radius in steps (Eq. chi_filtered)
    R_w: float = 1.0                  # temporal filter radius of the rotation angle in steps (Eq. psi_filtered)
    filter_R: float = 0.0             # density filter radius in design cells (Eq. filtering); <= 1 is identity
    beta: float = 0.0                 # Heaviside projection steepness (Eq. projection); 0 = identity
    eta: float = 0.5                  # projection threshold
    probe_lo: tuple = ()              # objective box O_target, inclusive lower corner
    probe_hi: tuple = ()              # exclusive upper corner
    direction: tuple = ()             # n of Eq. objective1
    phi_var: float = 0.0              # phi of Eq. objective1: weight of the variance V in J1 = E - phi V
    objective: str = "J1"             # "J1" (Eq. objective1) or "J2" (Eq. objective2, the oar)
    w_D: float = 0.0                  # weights of F_D and T in J2 = F_L + w_D F_D + w_T T (Eq. objective2)
    w_T: float = 0.0
    drag_span: float = 1.0            # x_2^max - x_2^min of F_D (cells)
    l_m: float = 1.0                  # moment arm l_m of T (cells)
    wall_velocity: dict = field(default_factory=dict)  # {(axis, side): vector}; side 0 = plane 0, 1 = plane n-1

    @property
    def d(self) -> int:
        return len(self.shape)

    @property
    def ext(self) -> tuple:
        """Design grid including the margin on both sides."""
        return tuple(n + 2 * self.margin for n in self.design)

    def center(self) -> np.ndarray:
        if self.base_center is not None:
            return np.asarray(self.base_center, dtype=np.float64)
        return (np.asarray(self.shape, dtype=np.float64) - 1.0) / 2.0

    def origin(self) -> np.ndarray:
        """X0 - xi^G: analysis coordinate of design index 0 (incl. margin) at zero offset (Eq. rigid_body_position, theta = 0)."""
        xi_g = (np.asarray(self.ext, dtype=np.float64) - 1.0) / 2.0
        return self.center() - xi_g


# ---------------------------------------------------------------------------------------------
# LKS forward step (Sec. 2.2)
# ---------------------------------------------------------------------------------------------


def central_diff(f, axis):
    """(f(x + e_axis) - f(x - e_axis)) / 2 with periodic wrap (the velocity gradient of the Inamuro equilibrium)."""
    return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / 2.0


def equilibrium(p, u, A, c, w):
    """All f_i^eq(x) of the Inamuro equilibrium with the velocity-gradient term (Sec. 2.2, Eq. for f_i^eq).

    f_i = w_i {3p + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u} + w_i A (du_b/dx_a + du_a/dx_b) c_a c_b.
    """
    d = u.shape[0]
    uu = sum(u[a] * u[a] for a in range(d))
    # S_ab = du_b/dx_a + du_a/dx_b
    G = [[central_diff(u[b], a) for b in range(d)] for a in range(d)]  # G[a][b] = d u_b / d x_a
    S = [[G[a][b] + G[b][a] for b in range(d)] for a in range(d)]
    feq = []
    for i in range(len(w)):
        cu = sum(c[i, a] * u[a] for a in range(d))
        grad = sum(S[a][b] * (c[i, a] * c[i, b]) for a in range(d) for b in range(d))
        feq.append(w[i] * (3.0 * p + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu) + w[i] * A * grad)
    return feq


def stream_moments(feq, c):
    """p*(x) = 1/3 sum_i f_i^eq(x - c_i), u*(x) = sum_i c_i f_i^eq(x - c_i) (Eqs. p_tmp, u_tmp), tau = 1 stream."""
    d = c.shape[1]
    axes = tuple(range(d))
    pstar = 0.0
    ustar = [0.0] * d
    for i, f in enumerate(feq):
        g = np.roll(f, shift=tuple(int(v) for v in c[i]), axis=axes)  # g(x) = f(x - c_i)
        pstar = pstar + g / 3.0
        for a in range(d):
            if c[i, a] != 0:
                ustar[a] = ustar[a] + c[i, a] * g
    return pstar, np.stack([np.broadcast_to(v, feq[0].shape) for v in ustar])


def wall_mask(prob: Problem):
    """Boolean mask of wall nodes and the imposed wall velocity field (Sec. 2.2: p, u imposed directly).

    Reading: the wall nodes are the first and last index planes of every non-periodic axis; u is set to
    that plane's velocity (later axes win where planes meet); p is not overwritten.
    """
    d = prob.d
    mask = np.zeros(prob.shape, dtype=bool)
    uw = np.zeros((d,) + prob.shape)
    for a in range(d):
        if prob.periodic[a]:
            continue
        for side, idx in ((0, 0), (1, prob.shape[a] - 1)):
            sl = [slice(None)] * d
            sl[a] = idx
            mask[tuple(sl)] = True
            vel = prob.wall_velocity.get((a, side), (0.0,) * d)
            for b in range(d):
                uw[(b,) + tuple(sl)] = vel[b]
    return mask, uw


def lks_step(p, u, kappa, uS, A, c, w, mask, uw):
    """One LKS step (n-1 -> n): Eqs. p_tmp, u_tmp, p and u with the implicit Brinkman update, then walls."""
    feq = equilibrium(p, u, A, c, w)
    pstar, ustar = stream_moments(feq, c)
    unew = (ustar + kappa * uS) / (1.0 + kappa)
    unew = np.where(mask, uw, unew)
    return pstar, unew


# ---------------------------------------------------------------------------------------------
# Grid separation mapping (Sec. 2.3, Eqs. kappa, u_s, rigid_body_position, rigid_body_velocity)
# ---------------------------------------------------------------------------------------------


def kernel_halfwidth(kernel: str) -> int:
    return 1 if kernel == "linear" else 2


def w1(r, kernel):
    """One-dimensional transfer weight w(r) (Sec. 2.3; 'linear' is the hat max(0, 1 - |r|) the configs ask for)."""
    if kernel == "cosine":
        return np.where(np.abs(np.real(r)) <= 2.0, 0.25 * (1.0 + np.cos(np.pi * r / 2.0)), 0.0)
    return np.where(np.abs(np.real(r)) <= 1.0, 1.0 - np.sign(np.real(r)) * r, 0.0)


def dw1(r, kernel):
    """dw/dr on the tap pieces used by ``axis_taps`` (for the hat: -1 on [0, 1), +1 on [-1, 0))."""
    if kernel == "cosine":
        return np.where(np.abs(np.real(r)) <= 2.0, -(np.pi / 8.0) * np.sin(np.pi * r / 2.0), 0.0)
    rr = np.real(r)
    return np.where((rr > 0.0) & (rr <= 1.0), -1.0, np.where((rr > -1.0) & (rr <= 0.0), 1.0, 0.0))


def fold(t, n, hw):
    """Fold a local coordinate on a periodic axis into one period [-hw, n - hw)."""
    shift = np.floor((np.real(t) + hw) / n) * n
    return t - shift


def axis_taps(x, o, n, ne, periodic, kernel):
    """Taps of the rigidly shifted design grid along one axis.

    For analysis nodes x (1-D integer array) and design-index origin o (analysis coordinate of design index 0),
    the local coordinate is t = x - o.  Returns (j, wgt, dwgt_do, valid) of shape (len(x), 2*hw): the design
    indices, their weights w(t - j), the derivatives of the weights with respect to o, and validity.
    The tap window is the piece that contains t from the left (i0 = ceil(t) - 1), so the position derivative is
    the one-sided derivative from the right in o (reading of the hat kernel at integer offsets).
    """
    hw = kernel_halfwidth(kernel)
    t = x.astype(np.float64) - o if not np.iscomplexobj(o) else x - o
    if periodic:
        t = fold(t, n, hw)
    i0 = np.ceil(np.real(t)).astype(np.int64) - 1
    ks = np.arange(-(hw - 1), hw + 1)
    j = i0[:, None] + ks[None, :]
    r = t[:, None] - j
    wgt = w1(r, kernel)
    dwgt = -dw1(r, kernel)  # d w(t - j) / d o = -w'(r)
    valid = (j >= 0) & (j < ne)
    wgt = np.where(valid, wgt, 0.0)
    dwgt = np.where(valid, dwgt, 0.0)
    return np.clip(j, 0, ne - 1), wgt, dwgt, valid


def map_gather(kref, o, prob: Problem, with_grad=False):
    """kappa(x) = sum_j W(x - x^ref_j) kappa^ref_j and C(x) = sum_j W(x - x^ref_j) (Eqs. kappa, u_s) by taps.

    x^ref_j = j + o for translation only (theta = 0) with unit design spacing.  Returns kappa, C and, with
    with_grad, d kappa / d o_a and d C / d o_a for every axis a.
    """
    d = prob.d
    taps = []
    for a in range(d):
        x = np.arange(prob.shape[a])
        taps.append(axis_taps(x, o[a], prob.shape[a], prob.ext[a], prob.periodic[a], prob.kernel))
    T = taps[0][0].shape[1]
    kappa = 0.0
    dk = [0.0] * d
    for combo in np.ndindex(*([T] * d)):
        # separable weight over axes, gathered design value
        idx = []
        wt = 1.0
        for a in range(d):
            sh = [1] * d
            sh[a] = prob.shape[a]
            idx.append(taps[a][0][:, combo[a]].reshape(sh))
            wt = wt * taps[a][1][:, combo[a]].reshape(sh)
        val = kref[tuple(np.broadcast_arrays(*idx))]
        kappa = kappa + wt * val
        if with_grad:
            for a in range(d):
                g = 1.0
                for b in range(d):
                    sh = [1] * d
                    sh[b] = prob.shape[b]
                    col = taps[b][2 if b == a else 1][:, combo[b]].reshape(sh)
                    g = g * col
                dk[a] = dk[a] + g * val
    # C is separable: product over axes of the summed valid weights
    C = 1.0
    dC = [1.0] * d
    for a in range(d):
        sh = [1] * d
        sh[a] = prob.shape[a]
        s = taps[a][1].sum(axis=1).reshape(sh)
        ds = taps[a][2].sum(axis=1).reshape(sh)
        C = C * s
        for b in range(d):
            dC[b] = dC[b] * (ds if b == a else s)
    kappa = np.broadcast_to(kappa, prob.shape)
    C = np.broadcast_to(C, prob.shape)
    if not with_grad:
        return kappa, C
    dk = [np.broadcast_to(v, prob.shape) for v in dk]
    dC = [np.broadcast_to(v, prob.shape) for v in dC]
    return kappa, C, dk, dC


def map_gather_T(gk, o, prob: Problem):
    """Transpose of the kappa mapping: g_j = sum_x W(x - x^ref_j) gk(x) (the scatter-add onto the design grid, Eq. dJdgamma)."""
    d = prob.d
    taps = []
    for a in range(d):
        x = np.arange(prob.shape[a])
        taps.append(axis_taps(x, o[a], prob.shape[a], prob.ext[a], prob.periodic[a], prob.kernel))
    T = taps[0][0].shape[1]
    out = np.zeros(prob.ext, dtype=np.result_type(gk, o, np.float64))
    for combo in np.ndindex(*([T] * d)):
        idx = []
        wt = 1.0
        for a in range(d):
            sh = [1] * d
            sh[a] = prob.shape[a]
            idx.append(taps[a][0][:, combo[a]].reshape(sh))
            wt = wt * taps[a][1][:, combo[a]].reshape(sh)
        np.add.at(out, tuple(np.broadcast_arrays(*idx)), np.broadcast_to(wt * gk, prob.shape))
    return out


def map_bruteforce(kref, o, prob: Problem):
    """The literal Eqs. kappa, u_s: for every analysis node, sum W over every design node (incl. margin).

    Periodic axes take the nearest periodic image of the displacement; on wall axes nothing is folded, so
    contributions that land outside the grid are dropped.  O(N * N_d): tiny grids only.
    """
    d = prob.d
    xs = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in prob.shape], indexing="ij"), axis=-1)
    js = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in prob.ext], indexing="ij"), axis=-1)
    X = xs.reshape(-1, d)
    Jc = js.reshape(-1, d) + np.asarray(o)[None, :]
    W = np.ones((X.shape[0], Jc.shape[0]))
    for a in range(d):
        r = X[:, a][:, None] - Jc[:, a][None, :]
        if prob.periodic[a]:
            n = prob.shape[a]
            r = r - n * np.round(r / n)
        W = W * w1(r, prob.kernel)
    kappa = (W @ kref.reshape(-1)).reshape(prob.shape)
    C = W.sum(axis=1).reshape(prob.shape)
    return kappa, C


# ---------------------------------------------------------------------------------------------
# Rigid rotation about an axis parallel to z (Sec. 2.3, Eqs. rigid_body_position, rigid_body_velocity, kappa,
# u_s; Sec. 2.5, the derivatives of x^ref and u^S,ref with respect to theta).  The rotated design lattice is no
# longer aligned with the analysis axes, so these functions write the mapping out as a dense weight matrix
# W[x, j] over every analysis node x and every node j of the extended design grid (tiny grids only).
# ---------------------------------------------------------------------------------------------


def rotation_matrix(theta):
    """R(theta) of Eq. rigid_body_position (acts on the x-y components)."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s], [s, c]])


def rotation_matrix_d(theta):
    """dR/dtheta: the matrix of Eq. rigid_body_velocity and of d x^ref / d theta."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[-s, -c], [c, -s]])


def rotation_matrix_dd(theta):
    """d^2R/dtheta^2: the matrix of d u^S,ref / d theta (per unit omega)."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[-c, s], [-s, -c]])


def design_arms(prob: Problem):
    """xi_j - xi^G for every node j of the extended design grid, shape (N_d, d), in the order of kref.reshape(-1)."""
    js = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in prob.ext], indexing="ij"), axis=-1)
    xi_g = (np.asarray(prob.ext, dtype=np.float64) - 1.0) / 2.0
    return js.reshape(-1, prob.d) - xi_g[None, :]


def rotated_reference(prob: Problem, o, theta):
    """x^ref_j = R(theta)(xi_j - xi^G) + x^G (Eq. rigid_body_position) and d x^ref_j / d theta, shape (N_d, d).

    o is the analysis coordinate of design index 0 at theta = 0 (so x^G = o + xi^G, and theta = 0 gives the
    translated lattice x^ref_j = j + o).  In 3D the rotation turns x and y about an axis parallel to z.
    """
    arm = design_arms(prob)
    xi_g = (np.asarray(prob.ext, dtype=np.float64) - 1.0) / 2.0
    dtype = np.result_type(theta, np.asarray(o), np.float64)
    xref = arm.astype(dtype)
    xref[:, :2] = arm[:, :2] @ rotation_matrix(theta).T
    xref = xref + (np.asarray(o) + xi_g)[None, :]
    dxref = np.zeros_like(xref)
    dxref[:, :2] = arm[:, :2] @ rotation_matrix_d(theta).T
    return xref, dxref


def weight_matrix(prob: Problem, xref):
    """W[x, j] = prod_a w(x_a - x^ref_{j,a}) (the weight function of Eqs. kappa, u_s) and dW/dx^ref_{j,a}.

    Periodic axes take the nearest periodic image of the displacement; on wall axes nothing is folded, so weight
    that lands outside the grid is dropped (as in ``map_bruteforce``).  Derivatives use ``dw1``'s pieces.
    """
    d = prob.d
    X = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in prob.shape], indexing="ij"),
                 axis=-1).reshape(-1, d)
    ws, dws = [], []
    for a in range(d):
        r = X[:, a][:, None] - xref[:, a][None, :]
        if prob.periodic[a]:
            n = prob.shape[a]
            r = r - n * np.round(np.real(r) / n)
        ws.append(w1(r, prob.kernel))
        dws.append(dw1(r, prob.kernel))
    W = ws[0]
    for a in range(1, d):
        W = W * ws[a]
    dW = []
    for a in range(d):
        g = -dws[a]  # d w(x - x^ref) / d x^ref = -w'(r)
        for b in range(d):
            if b != a:
                g = g * ws[b]
        dW.append(g)
    return W, dW


def map_rotated(kref, o, theta, omega, uG, prob: Problem, with_grad=False):
    """kappa(x) = sum_j W(x, x^ref_j) kappa^ref_j and u^S(x) = sum_j W(x, x^ref_j) u^S,ref_j (Eqs. kappa, u_s) for the
    rotated pose, u^S,ref_j = R'(theta)(xi_j - xi^G) omega + u^G (Eq. rigid_body_velocity).

    Returns kappa (shape), u^S (d, shape) and, with_grad, a dict of the derivatives with respect to o_a (= x^G_a),
    theta, omega and u^G_a (the last is C = sum_j W, the same for every component), plus W itself.
    """
    d = prob.d
    xref, dxref = rotated_reference(prob, o, theta)
    W, dW = weight_matrix(prob, xref)
    arm = design_arms(prob)
    kr = kref.reshape(-1)
    dtype = np.result_type(W, theta, omega, uG, np.float64)
    vref = np.zeros((arm.shape[0], d), dtype=dtype)
    vref[:, :2] = (arm[:, :2] @ rotation_matrix_d(theta).T) * omega
    vref = vref + np.asarray(uG)[None, :]
    shp = prob.shape
    kappa = (W @ kr).reshape(shp)
    uS = np.stack([(W @ vref[:, b]).reshape(shp) for b in range(d)])
    if not with_grad:
        return kappa, uS
    dWdth = sum(dW[a] * dxref[:, a][None, :] for a in range(d))
    dv_dth = np.zeros_like(vref)
    dv_dth[:, :2] = (arm[:, :2] @ rotation_matrix_dd(theta).T) * omega
    dv_dom = np.zeros_like(vref)
    dv_dom[:, :2] = arm[:, :2] @ rotation_matrix_d(theta).T
    G = {
        "W": W,
        "dk_do": [(dW[a] @ kr).reshape(shp) for a in range(d)],
        "dk_dth": (dWdth @ kr).reshape(shp),
        "duS_do": [[(dW[a] @ vref[:, b]).reshape(shp) for b in range(d)] for a in range(d)],
        "duS_dth": [(dWdth @ vref[:, b] + W @ dv_dth[:, b]).reshape(shp) for b in range(d)],
        "duS_dom": [(W @ dv_dom[:, b]).reshape(shp) for b in range(d)],
        "C": W.sum(axis=1).reshape(shp),
    }
    return kappa, uS, G


# ---------------------------------------------------------------------------------------------
# Shape parametrisation (Sec. 3.1, Eqs. filtering, projection; Sec. 2.3, Eq. kappa_ref)
# ---------------------------------------------------------------------------------------------


def filter_weights(shape, R):
    """Dense matrix of cone weights w_s(x_i, x_j) = max(0, (R - |x_i - x_j|)/R) over the design grid (Eq. filtering)."""
    pts = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij"), -1).reshape(-1, len(shape))
    dist = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    return np.maximum(0.0, (R - dist) / R)


def density_filter(gamma, R):
    """gamma~_i = sum_j w_s gamma_j / sum_j w_s, truncated normalisation at the edges (Eq. filtering)."""
    if R <= 1.0:
        return gamma.copy()
    out = np.zeros_like(gamma)
    r = int(math.floor(R))
    shape = gamma.shape
    norm = np.zeros(shape)
    for off in np.ndindex(*([2 * r + 1] * gamma.ndim)):
        dvec = np.array(off) - r
        dist = math.sqrt(float((dvec * dvec).sum()))
        wgt = max(0.0, (R - dist) / R)
        if wgt == 0.0:
            continue
        src, dst = [], []
        for a, dv in enumerate(dvec):
            n = shape[a]
            dst.append(slice(max(0, -dv), min(n, n - dv)))
            src.append(slice(max(0, dv), min(n, n + dv)))
        out[tuple(dst)] += wgt * gamma[tuple(src)]
        norm[tuple(dst)] += wgt
    return out / norm


def density_filter_T(g, R):
    """Transpose of ``density_filter``: dJ/dgamma_j = sum_i w_s(i, j) (dJ/dgamma~_i) / sum_k w_s(i, k)."""
    if R <= 1.0:
        return g.copy()
    # row norms of the filter, then the transposed weighted sum
    r = int(math.floor(R))
    shape = g.shape
    norm = np.zeros(shape)
    for off in np.ndindex(*([2 * r + 1] * g.ndim)):
        dvec = np.array(off) - r
        wgt = max(0.0, (R - math.sqrt(float((dvec * dvec).sum()))) / R)
        if wgt == 0.0:
            continue
        src, dst = [], []
        for a, dv in enumerate(dvec):
            n = shape[a]
            dst.append(slice(max(0, -dv), min(n, n - dv)))
            src.append(slice(max(0, dv), min(n, n + dv)))
        norm[tuple(dst)] += wgt
    h = g / norm
    out = np.zeros_like(h)
    for off in np.ndindex(*([2 * r + 1] * g.ndim)):
        dvec = np.array(off) - r
        wgt = max(0.0, (R - math.sqrt(float((dvec * dvec).sum()))) / R)
        if wgt == 0.0:
            continue
        src, dst = [], []
        for a, dv in enumerate(dvec):
            n = shape[a]
            dst.append(slice(max(0, -dv), min(n, n - dv)))
            src.append(slice(max(0, dv), min(n, n + dv)))
        # the forward sent gamma_j (src) to gamma~_i (dst); the transpose sends h_i back to j
        out[tuple(src)] += wgt * h[tuple(dst)]
    return out


def projection(gt, beta, eta):
    """Heaviside projection (Eq. projection); beta = 0 is the identity (its beta -> 0 limit)."""
    if beta == 0.0:
        return gt.copy()
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return (np.tanh(beta * eta) + np.tanh(beta * (gt - eta))) / den


def projection_deriv(gt, beta, eta):
    """d gamma-bar / d gamma~ of Eq. projection."""
    if beta == 0.0:
        return np.ones_like(gt)
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return beta / np.cosh(beta * (gt - eta)) ** 2 / den


def kappa_ref(gb, kappa_max, q):
    """kappa^ref = kappa_max q gamma / ((1 - gamma) + q) (Eq. kappa_ref)."""
    return kappa_max * q * gb / ((1.0 - gb) + q)


def kappa_ref_deriv(gb, kappa_max, q):
    return kappa_max * q * (1.0 + q) / ((1.0 - gb) + q) ** 2


def embed_margin(a, margin):
    """Place the inner design array inside the extended grid with a zero (fluid) margin (Sec. 2.3)."""
    return np.pad(a, margin, mode="constant")


def strip_margin(a, margin):
    sl = tuple(slice(margin, n - margin) for n in a.shape)
    return a[sl]


# ---------------------------------------------------------------------------------------------
# Motion parametrisation (Sec. 2.4, Eqs. chi_filtered, x_g, u_g)
# ---------------------------------------------------------------------------------------------


def knot_times(K, Nt):
    """Knot k sits at step k Nt / (K - 1) (reading of the knot representation of chi(t))."""
    return np.arange(K, dtype=np.float64) * Nt / (K - 1)


def temporal_filter_matrix(K, Nt, R_t):
    """Normalised triangular weights of Eq. chi_filtered evaluated between knot times (truncated, non-periodic)."""
    tk = knot_times(K, Nt)
    W = np.maximum(0.0, (R_t - np.abs(tk[:, None] - tk[None, :])) / R_t)
    return W / W.sum(axis=1, keepdims=True)


def motion_filter(knots, Nt, R_t):
    """Filtered knot positions chi~ (Eq. chi_filtered); knots has shape (K, d)."""
    return temporal_filter_matrix(knots.shape[0], Nt, R_t) @ knots


def motion_filter_T(g, Nt, R_t):
    return temporal_filter_matrix(g.shape[0], Nt, R_t).T @ g


def interp_matrix(K, Nt):
    """Linear interpolation of knot values to every step n = 0..Nt (integer arithmetic for the segment index)."""
    M = np.zeros((Nt + 1, K))
    for n in range(Nt + 1):
        num = n * (K - 1)
        k = min(num // Nt, K - 2)
        th = (num - k * Nt) / Nt
        M[n, k] += 1.0 - th
        M[n, k + 1] += th
    return M


def angles(aknots, Nt, R_w):
    """Per-step rotation angle theta_n and angular velocity omega_n = theta_n - theta_{n-1} (Eqs. psi_filtered, theta,
    omega): the angle knots (radians, shape (K_w,)) are filtered and interpolated like the position knots."""
    th = interp_matrix(len(aknots), Nt) @ motion_filter(np.asarray(aknots)[:, None], Nt, R_w)[:, 0]
    om = np.zeros_like(th)
    om[1:] = th[1:] - th[:-1]
    om[0] = om[1]
    return th, om


def positions(knots, Nt, R_t):
    """Per-step offsets s_n (n = 0..Nt) and velocities u^G_n = s_n - s_{n-1} (Eq. u_g, backward difference)."""
    s = interp_matrix(knots.shape[0], Nt) @ motion_filter(knots, Nt, R_t)
    uG = np.zeros_like(s)
    uG[1:] = s[1:] - s[:-1]
    uG[0] = uG[1]
    return s, uG


# ---------------------------------------------------------------------------------------------
# Forward solve, objective and exact discrete adjoint (Sec. 2.2, 2.5, 2.6; Algorithm 1)
# ---------------------------------------------------------------------------------------------


def probe_weights(prob: Problem):
    """phi(x) = n 1_O(x) / (Nt |O|): d E / d u_n(x) for every step n >= 1 (E of Eq. objective1).

    O excludes wall nodes.
    """
    box = probe_mean_weights(prob)
    phi = np.zeros((prob.d,) + prob.shape)
    for a in range(prob.d):
        phi[a] = box * prob.direction[a]
    return phi


def probe_mean_weights(prob: Problem):
    """1_O(x) / (Nt |O|): the weight of one node and step in the space-time means of Eq. objective1."""
    mask, _ = wall_mask(prob)
    box = np.zeros(prob.shape, dtype=bool)
    box[tuple(slice(lo, hi) for lo, hi in zip(prob.probe_lo, prob.probe_hi))] = True
    box &= ~mask
    count = int(box.sum())
    return np.where(box, 1.0, 0.0) / (prob.Nt * count)


def flow_along(prob: Problem, u):
    """n . u at every node (the integrand of E in Eq. objective1)."""
    return sum(prob.direction[a] * u[a] for a in range(prob.d))


def objective_source(prob: Problem, phi, E, u):
    """d J1 / d u_n(x) for J1 = E - phi_V V (Eq. objective1), V = S2 - E^2 with S2 the mean of (n.u)^2:
    phi(x) [1 + 2 phi_V E - 2 phi_V n.u_n(x)].  E is the mean of the whole forward run."""
    if prob.phi_var == 0.0:
        return phi
    return phi * (1.0 + 2.0 * prob.phi_var * E - 2.0 * prob.phi_var * flow_along(prob, u))


def design_mask(prob: Problem):
    """The inner design grid D inside the extended one (the margin is fluid and not part of D)."""
    m = np.zeros(prob.ext, dtype=bool)
    m[tuple(slice(prob.margin, prob.margin + n) for n in prob.design)] = True
    return m


def oar_force_weights(prob: Problem, r, omega, uG):
    """g_{j,b} = d j2_n / d F_{j,b} for the Brinkman force density F_j = kappa^ref_j (u^ref_j - u^S,ref_j) of step n
    (Eq. objective2 read as a rectangle rule over n = 1..Nt): F_L weighs F_1 by 1/(Nt |D|), w_D F_D weighs F_2 by
    w_D u^G_2 / ((x_2^max - x_2^min) |D|), w_T T weighs e_3ab r_a F_b (r = x^ref - x^G) by w_T omega / (2 pi l_m |D|)."""
    nD = float(np.prod(prob.design))
    cL = 1.0 / (prob.Nt * nD)
    cD = prob.w_D / (prob.drag_span * nD)
    cT = prob.w_T / (2.0 * np.pi * prob.l_m * nD)
    inD = design_mask(prob).reshape(-1)
    g = np.zeros(r.shape, dtype=np.result_type(r, omega, uG, np.float64))
    g[:, 0] = np.where(inD, cL - cT * omega * r[:, 1], 0.0)
    g[:, 1] = np.where(inD, cD * uG[1] + cT * omega * r[:, 0], 0.0)
    return g, cD, cT, inD


def oar_terms(prob: Problem, kref, u, o, theta, omega, uG):
    """(F_L, F_D, T) integrands of step n of Eq. objective2 (already divided by their normalisations): u^ref_j is the
    transposed-mapped velocity sum_x W(x, x^ref_j) u(x), u^S,ref_j that of Eq. rigid_body_velocity."""
    xref, _ = rotated_reference(prob, o, theta)
    W, _ = weight_matrix(prob, xref)
    arm = design_arms(prob)
    d = prob.d
    U = np.stack([W.T @ u[b].reshape(-1) for b in range(d)], axis=1)
    v = np.zeros_like(U)
    v[:, :2] = (arm[:, :2] @ rotation_matrix_d(theta).T) * omega
    v = v + np.asarray(uG)[None, :]
    F = kref.reshape(-1)[:, None] * (U - v)
    r = xref - (np.asarray(o) + (np.asarray(prob.ext, dtype=np.float64) - 1.0) / 2.0)[None, :]
    nD = float(np.prod(prob.design))
    inD = design_mask(prob).reshape(-1)
    FL = np.where(inD, F[:, 0], 0.0).sum() / (prob.Nt * nD)
    FD = uG[1] * np.where(inD, F[:, 1], 0.0).sum() / (prob.drag_span * nD)
    T = omega * np.where(inD, r[:, 0] * F[:, 1] - r[:, 1] * F[:, 0], 0.0).sum() / (2.0 * np.pi * prob.l_m * nD)
    return FL, FD, T


def oar_step(prob: Problem, kref, u, o, theta, omega, uG, with_grad=False):
    """j2_n = F_L + w_D F_D + w_T T of step n (Eq. objective2) and, with_grad, its partial derivatives: dJ/du_n (the
    adjoint source, (d,) + shape), dJ/dkref (explicit, extended grid), dJ/do (= dJ/dx^G), dJ/du^G, dJ/dtheta, dJ/domega."""
    FL, FD, T = oar_terms(prob, kref, u, o, theta, omega, uG)
    j2 = FL + prob.w_D * FD + prob.w_T * T
    if not with_grad:
        return j2
    d = prob.d
    xref, dxref = rotated_reference(prob, o, theta)
    W, dW = weight_matrix(prob, xref)
    arm = design_arms(prob)
    kr = kref.reshape(-1)
    U = np.stack([W.T @ u[b].reshape(-1) for b in range(d)], axis=1)
    R1 = arm[:, :2] @ rotation_matrix_d(theta).T   # d u^S,ref / d omega (x-y components), also d r / d theta
    R2 = arm[:, :2] @ rotation_matrix_dd(theta).T  # d^2 r / d theta^2
    v = np.zeros_like(U)
    v[:, :2] = R1 * omega
    v = v + np.asarray(uG)[None, :]
    F = kr[:, None] * (U - v)
    r = xref - (np.asarray(o) + (np.asarray(prob.ext, dtype=np.float64) - 1.0) / 2.0)[None, :]
    g, cD, cT, inD = oar_force_weights(prob, r, omega, uG)
    gU = g * kr[:, None]           # d j2 / d u^ref_{j,b}
    src = np.stack([(W @ gU[:, b]).reshape(prob.shape) for b in range(d)])
    g_kref = (g * (U - v)).sum(axis=1).reshape(prob.ext)
    gv = -gU                       # d j2 / d u^S,ref_{j,b}
    g_uG = gv.sum(axis=0)
    g_uG[1] = g_uG[1] + cD * np.where(inD, F[:, 1], 0.0).sum()
    g_om = (gv[:, :2] * R1).sum() + cT * np.where(inD, r[:, 0] * F[:, 1] - r[:, 1] * F[:, 0], 0.0).sum()
    g_th = (gv[:, :2] * R2).sum() * omega
    # u^ref moves with x^ref
    gx = np.stack([sum(gU[:, b] * (dW[a].T @ u[b].reshape(-1)) for b in range(d)) for a in range(d)], axis=1)
    g_o = gx.sum(axis=0)
    g_th = g_th + (gx * dxref).sum()
    # the torque arm r = R(theta)(xi - xi^G)
    g_th = g_th + (cT * omega * np.where(inD, F[:, 1] * dxref[:, 0] - F[:, 0] * dxref[:, 1], 0.0)).sum()
    return j2, src, g_kref, g_o, g_uG, g_th, g_om


def initial_state(prob: Problem, dtype=np.float64):
    """p = 1/3, u = 0 everywhere, wall nodes at their wall velocity (Sec. 4 initial conditions)."""
    mask, uw = wall_mask(prob)
    p = np.full(prob.shape, 1.0 / 3.0, dtype=dtype)
    u = np.where(mask[None], uw, 0.0).astype(dtype)
    return p, u


def forward(prob: Problem, kref, s, uG, store=False, state0=None, rot=None):
    """Run Nt LKS steps (Algorithm 1, forward loop) and return J1 = E - phi_V V (Eq. objective1), or J2 (Eq.
    objective2, ``oar_step`` summed over n = 1..Nt) when prob.objective is "J2".

    E and S2 are rectangle-rule means over n = 1..Nt and the fluid nodes of O_target of n.u and (n.u)^2;
    V = S2 - E^2.

    kref is the extended design array kappa^ref (margin included); s, uG are (Nt+1, d) offsets and velocities;
    rot = (theta, omega), each (Nt+1,), turns the body (``map_rotated``); None keeps theta = 0 (``map_gather``).
    With store=True the list of states (p_n, u_n), n = 0..Nt, is returned too.
    """
    c, w = lattice(prob.lattice)
    A = viscosity_A(prob.nu)
    mask, uw = wall_mask(prob)
    phi = probe_weights(prob)
    wO = probe_mean_weights(prob)
    o0 = prob.origin()
    dtype = np.result_type(kref, s, uG, np.float64)
    p, u = initial_state(prob, dtype) if state0 is None else state0
    states = [(p, u)] if store else None
    E = 0.0
    S2 = 0.0
    J2 = 0.0
    for n in range(1, prob.Nt + 1):
        o = o0 + s[n]
        if rot is None:
            kappa, C = map_gather(kref, o, prob)
            uS = np.stack([uG[n, a] * C for a in range(prob.d)])
        else:
            kappa, uS = map_rotated(kref, o, rot[0][n], rot[1][n], uG[n], prob)
        p, u = lks_step(p, u, kappa, uS, A, c, w, mask, uw)
        if prob.objective == "J2":
            th, om = (0.0, 0.0) if rot is None else (rot[0][n], rot[1][n])
            J2 = J2 + oar_step(prob, kref, u, o, th, om, uG[n])
        E = E + (phi * u).sum()
        if prob.phi_var != 0.0:
            S2 = S2 + (wO * flow_along(prob, u) ** 2).sum()
        if store:
            states.append((p, u))
    J = E if prob.phi_var == 0.0 else E - prob.phi_var * (S2 - E * E)
    if prob.objective == "J2":
        J = J2
    return (J, states) if store else J


def adjoint(prob: Problem, kref, s, uG, states, rot=None, terminal=None, lambda0=None):
    """Exact discrete adjoint of ``forward`` (reverse sweep of Algorithm 1; discrete form of Eqs. ap_tmp-as).

    Returns dJ/dkref (extended grid), dJ/ds_n and dJ/du^G_n for n = 0..Nt (row 0 is zero).
    Per step n, going backward, with lam = dJ/d(p_n, u_n):
      b3  u-bar* = lam_u / (1 + kappa) off the walls, 0 on them; p-bar* = lam_p;
          kappa-bar = lam_u . (u^S - u_n) / (1 + kappa);  u^S-bar = lam_u kappa / (1 + kappa)
      b1  F-bar_i(y) = p-bar*(y + c_i) / 3 + c_i . u-bar*(y + c_i); moments M0, M1, M2 with weights w_i
      b2  lam_p(n-1) = 3 M0;  lam_u(n-1) = 3 M1 + 9 M2 u_{n-1} - 3 u_{n-1} M0
                       + A sum_a [M2_a.(y - e_a) - M2_a.(y + e_a)]  (+ dJ/du_{n-1} for n - 1 >= 1)
      b4  dJ/dkref += M^T kappa-bar (transposed mapping)
      b5  dJ/ds_n = sum_x kappa-bar dkappa/ds + (u^S-bar . u^G) dC/ds;  dJ/du^G_n = sum_x u^S-bar C
    The objective's own source dJ/du_n (``objective_source``) uses the mean E of the stored forward run.
    With rot = (theta, omega) (``forward``'s rotated pose) b4 and b5 go through the dense ``map_rotated``, and
    dJ/dtheta_n = sum_x kappa-bar dkappa/dtheta + u^S-bar . du^S/dtheta, dJ/domega_n = sum_x u^S-bar . du^S/domega
    are returned as two more (Nt+1,) arrays.
    terminal = (lam_p, lam_u) is added to the terminal adjoint state (the periodic approximation of Sec. 3.3 passes
    the previous iteration's lambda_0 there); with a list as lambda0, (lam_p, lam_u) at n = 0 is appended to it.
    """
    c, w = lattice(prob.lattice)
    A = viscosity_A(prob.nu)
    mask, _ = wall_mask(prob)
    phi = probe_weights(prob)
    E = sum((phi * states[n][1]).sum() for n in range(1, prob.Nt + 1))
    d = prob.d
    axes = tuple(range(d))
    o0 = prob.origin()
    dtype = np.result_type(kref, s, uG, np.float64)
    oar = prob.objective == "J2"

    def oar_at(m):
        th, om = (0.0, 0.0) if rot is None else (rot[0][m], rot[1][m])
        return oar_step(prob, kref, states[m][1], o0 + s[m], th, om, uG[m], with_grad=True)

    lam_p = np.zeros(prob.shape, dtype=dtype)
    if oar:
        src_next = oar_at(prob.Nt)
        lam_u = src_next[1].astype(dtype)
    else:
        lam_u = objective_source(prob, phi, E, states[prob.Nt][1]).astype(dtype)
    if terminal is not None:
        lam_p = lam_p + terminal[0]
        lam_u = lam_u + terminal[1]
    g_kref = np.zeros(prob.ext, dtype=dtype)
    g_s = np.zeros((prob.Nt + 1, d), dtype=dtype)
    g_uG = np.zeros((prob.Nt + 1, d), dtype=dtype)
    g_th = np.zeros(prob.Nt + 1, dtype=dtype)
    g_om = np.zeros(prob.Nt + 1, dtype=dtype)
    for n in range(prob.Nt, 0, -1):
        o = o0 + s[n]
        if oar:
            # explicit dependences of step n's oar integrand (its u_n source is already in lam_u)
            _, _, gk2, go2, guG2, gth2, gom2 = src_next
            g_kref = g_kref + gk2
            g_s[n] = g_s[n] + go2
            g_uG[n] = g_uG[n] + guG2
            g_th[n] = g_th[n] + gth2
            g_om[n] = g_om[n] + gom2
        if rot is None:
            kappa, C, dk, dC = map_gather(kref, o, prob, with_grad=True)
            uS = np.stack([uG[n, a] * C for a in range(d)])
        else:
            kappa, uS, G = map_rotated(kref, o, rot[0][n], rot[1][n], uG[n], prob, with_grad=True)
        u_n = states[n][1]
        u_prev = states[n - 1][1]
        # b3: Brinkman and wall adjoint, local sensitivities
        ubar = np.where(mask[None], 0.0, lam_u / (1.0 + kappa))
        pbar = lam_p
        kbar = np.where(mask, 0.0, sum(lam_u[a] * (uS[a] - u_n[a]) for a in range(d)) / (1.0 + kappa))
        uSbar = np.where(mask[None], 0.0, lam_u * kappa / (1.0 + kappa))
        # b4, b5
        if rot is None:
            g_kref = g_kref + map_gather_T(kbar, o, prob)
            Cbar = sum(uSbar[a] * uG[n, a] for a in range(d))
            for a in range(d):
                g_s[n, a] += (kbar * dk[a]).sum() + (Cbar * dC[a]).sum()
                g_uG[n, a] += (uSbar[a] * C).sum()
        else:
            g_kref = g_kref + (G["W"].T @ kbar.reshape(-1)).reshape(prob.ext)
            for a in range(d):
                g_s[n, a] += (kbar * G["dk_do"][a]).sum() + sum((uSbar[b] * G["duS_do"][a][b]).sum() for b in range(d))
                g_uG[n, a] += (uSbar[a] * G["C"]).sum()
            g_th[n] += (kbar * G["dk_dth"]).sum() + sum((uSbar[b] * G["duS_dth"][b]).sum() for b in range(d))
            g_om[n] += sum((uSbar[b] * G["duS_dom"][b]).sum() for b in range(d))
        # b1: reverse stream and local moments
        M0 = 0.0
        M1 = [0.0] * d
        M2 = [[0.0] * d for _ in range(d)]
        for i in range(len(w)):
            sh = tuple(-int(v) for v in c[i])  # g(y) = h(y + c_i)
            Fb = np.roll(pbar, shift=sh, axis=axes) / 3.0
            for a in range(d):
                if c[i, a] != 0:
                    Fb = Fb + c[i, a] * np.roll(ubar[a], shift=sh, axis=axes)
            M0 = M0 + w[i] * Fb
            for a in range(d):
                M1[a] = M1[a] + w[i] * c[i, a] * Fb
                for b in range(d):
                    M2[a][b] = M2[a][b] + w[i] * c[i, a] * c[i, b] * Fb
        # b2: adjoint of the equilibrium (pressure, quadratic and velocity-gradient terms)
        new_p = 3.0 * M0
        new_u = []
        for b in range(d):
            v = 3.0 * M1[b] - 3.0 * u_prev[b] * M0
            for a in range(d):
                v = v + 9.0 * M2[a][b] * u_prev[a]
                v = v + A * (np.roll(M2[a][b], 1, axis=a) - np.roll(M2[a][b], -1, axis=a))
            new_u.append(v)
        lam_p = new_p
        lam_u = np.stack(new_u)
        if n - 1 >= 1:
            if oar:
                src_next = oar_at(n - 1)
                lam_u = lam_u + src_next[1]
            else:
                lam_u = lam_u + objective_source(prob, phi, E, u_prev)
    if lambda0 is not None:
        lambda0.append((lam_p, lam_u))
    if rot is not None:
        return g_kref, g_s, g_uG, g_th, g_om
    return g_kref, g_s, g_uG


# ---------------------------------------------------------------------------------------------
# Full problem: design variables -> J and gradients (Algorithm 1: filters, forward, adjoint, chain rule)
# ---------------------------------------------------------------------------------------------


# ---------------------------------------------------------------------------------------------
# The paper's continuous adjoint, the ALKS (Sec. 2.5, Eqs. ap_tmp-as), as an alternative to ``adjoint``
# ---------------------------------------------------------------------------------------------


def adjoint_alks(prob: Problem, kref, s, uG, states):
    """Reverse sweep of the ALKS (Sec. 2.5) for J1 with phi_V = 0, and its sensitivities (Eqs. dJdgamma, dJdchi).

    Adjoint moments (p~, u~, s~) at step n; going from n to n-1:
      f~eq_i(z) = p~ + 3 c_ia (u~_a + 3 s~_ab u_b - p~ u_a) - A c_ia d_b(s~_ab + s~_ba), everything at node z and
                  step n (u the state of step n, d_b the central difference);
      p~*, u~*, s~* at node x and step n-1 = sum_i w_i {1, c_i, c_i c_i} f~eq_i(x + c_i)           (Eqs. ap_tmp-as_tmp)
      sources at step n-1 (Eqs. ap-as): the Brinkman term -3 kappa c_ib u~_b makes u~ implicit, u~ (1 + kappa) =
      u~* - sum_i w_i c_i dJ/df_i with dJ/df_i = c_i . n / (Nt |O|) on the probe nodes (its p~ and s~ moments vanish
      by symmetry), so u~ = (u~* - n / (3 Nt |O|)) / (1 + kappa); u~ = 0 on wall nodes, where u is imposed.
    The terminal state (step Nt) is the source alone.  The sensitivities are the ALKS forms: kappa-bar = 3 (u_n -
    u^S_n) . u~_n and u^S-bar = -3 kappa_n u~_n, taken through the same transposed mapping and position derivatives as
    in ``adjoint``.  Returns (dJ/dkref, dJ/ds_n, dJ/du^G_n) like ``adjoint``.
    Readings: u in f~eq is the state at the same step and node as the adjoint moments; the walls are handled as in
    the forward (u~ imposed to 0 there, p~ and s~ streamed).
    """
    c, w = lattice(prob.lattice)
    A = viscosity_A(prob.nu)
    mask, _ = wall_mask(prob)
    phi = probe_weights(prob)
    d = prob.d
    axes = tuple(range(d))
    o0 = prob.origin()
    dtype = np.result_type(kref, s, uG, np.float64)

    def brinkman(ustar_src, kappa):
        return np.where(mask[None], 0.0, ustar_src / (1.0 + kappa))

    kappa_n, C_n = map_gather(kref, o0 + s[prob.Nt], prob)
    pt = np.zeros(prob.shape, dtype=dtype)
    st = np.zeros((d, d) + prob.shape, dtype=dtype)
    ut = brinkman(-phi / 3.0, kappa_n).astype(dtype)
    g_kref = np.zeros(prob.ext, dtype=dtype)
    g_s = np.zeros((prob.Nt + 1, d), dtype=dtype)
    g_uG = np.zeros((prob.Nt + 1, d), dtype=dtype)
    for n in range(prob.Nt, 0, -1):
        o = o0 + s[n]
        kappa, C, dk, dC = map_gather(kref, o, prob, with_grad=True)
        u_n = states[n][1]
        uS = np.stack([uG[n, a] * C for a in range(d)])
        # sensitivities of step n (Eqs. dJdgamma, dJdchi in the notation of ``adjoint``)
        kbar = np.where(mask, 0.0, 3.0 * sum((u_n[a] - uS[a]) * ut[a] for a in range(d)))
        uSbar = np.where(mask[None], 0.0, -3.0 * kappa * ut)
        g_kref = g_kref + map_gather_T(kbar, o, prob)
        Cbar = sum(uSbar[a] * uG[n, a] for a in range(d))
        for a in range(d):
            g_s[n, a] = (kbar * dk[a]).sum() + (Cbar * dC[a]).sum()
            g_uG[n, a] = (uSbar[a] * C).sum()
        # f~eq at every node from the moments and the state of step n
        div = [sum(central_diff(st[a][b] + st[b][a], b) for b in range(d)) for a in range(d)]
        pstar = np.zeros_like(pt)
        ustar = np.zeros_like(ut)
        sstar = np.zeros_like(st)
        for i in range(len(w)):
            feq = pt.copy()
            for a in range(d):
                if c[i, a] != 0:
                    inner = ut[a] + 3.0 * sum(st[a][b] * u_n[b] for b in range(d)) - pt * u_n[a]
                    feq = feq + c[i, a] * (3.0 * inner - A * div[a])
            g = np.roll(feq, shift=tuple(-int(v) for v in c[i]), axis=axes)  # value at x + c_i
            pstar = pstar + w[i] * g
            for a in range(d):
                ustar[a] = ustar[a] + w[i] * c[i, a] * g
                for b in range(d):
                    sstar[a][b] = sstar[a][b] + w[i] * c[i, a] * c[i, b] * g
        pt, st = pstar, sstar
        if n - 1 >= 1:
            kappa_m, _ = map_gather(kref, o0 + s[n - 1], prob)
            ut = brinkman(ustar - phi / 3.0, kappa_m)
        else:
            ut = ustar
    return g_kref, g_s, g_uG


def gradient_alks(prob: Problem, gamma, knots):
    """``gradient`` with the ALKS sweep in place of the exact discrete adjoint."""
    kref, gt, gb = design_to_kref(prob, gamma)
    s, uG = positions(knots, prob.Nt, prob.R_t)
    J, states = forward(prob, kref, s, uG, store=True)
    g_kref, g_s, g_uG = adjoint_alks(prob, kref, s, uG, states)
    g_kr = strip_margin(g_kref, prob.margin)
    g_gb = g_kr * kappa_ref_deriv(gb, prob.kappa_max, prob.q)
    g_gt = g_gb * projection_deriv(gt, prob.beta, prob.eta)
    return J, density_filter_T(g_gt, prob.filter_R), knot_gradient(prob, g_s, g_uG), g_s, g_uG


# ---------------------------------------------------------------------------------------------
# Constraint functionals (Sec. 2.6, Eqs. constraint1, constraint2, constraint3)
# ---------------------------------------------------------------------------------------------


def solid_volume(gamma, V_max):
    """G1 = sum_D gamma / (V_max |D|) - 1 and dG1/dgamma (Eq. constraint1; D the inner design grid)."""
    n = gamma.size
    return gamma.sum() / (V_max * n) - 1.0, np.full(gamma.shape, 1.0 / (V_max * n))


def fluid_volume(gamma, V_max):
    """G2 = sum_D (1 - gamma) / (V_max |D|) - 1 and dG2/dgamma (Eq. constraint2)."""
    n = gamma.size
    return (1.0 - gamma).sum() / (V_max * n) - 1.0, np.full(gamma.shape, -1.0 / (V_max * n))


def angular_speed_bound(omega, omega_max, p):
    """G3 = (sum_n (omega_n / omega_max)^p)^(1/p) - 1 over n = 1..Nt (Eq. constraint3, rectangle rule, unit step)
    and dG3/domega_n (row 0 is zero: omega_0 enters no step)."""
    r = omega[1:] / omega_max
    S = (r ** p).sum()
    g = np.zeros_like(omega)
    g[1:] = S ** (1.0 / p - 1.0) * r ** (p - 1) / omega_max
    return S ** (1.0 / p) - 1.0, g


def design_to_kref(prob: Problem, gamma):
    """gamma -> gamma~ (filter) -> gamma-bar (projection) -> kappa^ref on the extended grid (Algorithm 1, first line)."""
    gt = density_filter(gamma, prob.filter_R)
    gb = projection(gt, prob.beta, prob.eta)
    kr = kappa_ref(gb, prob.kappa_max, prob.q)
    return embed_margin(kr, prob.margin), gt, gb


def solve(prob: Problem, gamma, knots, store=False, aknots=None):
    """J(gamma, knots) of the whole chain; aknots (angle knots in radians) turn the body (Sec. 2.4)."""
    kref, _, _ = design_to_kref(prob, gamma)
    s, uG = positions(knots, prob.Nt, prob.R_t)
    rot = None if aknots is None else angles(aknots, prob.Nt, prob.R_w)
    return forward(prob, kref, s, uG, store=store, rot=rot)


def knot_gradient(prob: Problem, g_s, g_uG):
    """Chain rule from per-step (dJ/ds_n, dJ/du^G_n) to the knots: difference^T, interpolation^T, filter^T."""
    gs = g_s.copy()
    gs[1:] += g_uG[1:]
    gs[:-1] -= g_uG[1:]
    # u^G_0 = u^G_1 is never used by a step, so g_uG[0] is zero
    gf = interp_matrix(prob.K, prob.Nt).T @ gs
    return motion_filter_T(gf, prob.Nt, prob.R_t)


def angle_gradient(prob: Problem, g_th, g_om, K_w):
    """Chain rule from per-step (dJ/dtheta_n, dJ/domega_n) to the angle knots (the same steps as ``knot_gradient``)."""
    gt = g_th.copy()
    gt[1:] += g_om[1:]
    gt[:-1] -= g_om[1:]
    gf = interp_matrix(K_w, prob.Nt).T @ gt
    return motion_filter_T(gf[:, None], prob.Nt, prob.R_w)[:, 0]


def gradient(prob: Problem, gamma, knots, aknots=None):
    """Return J, dJ/dgamma (inner design grid), dJ/dknots (K, d) and, with angle knots, dJ/daknots (K_w,)."""
    kref, gt, gb = design_to_kref(prob, gamma)
    s, uG = positions(knots, prob.Nt, prob.R_t)
    rot = None if aknots is None else angles(aknots, prob.Nt, prob.R_w)
    J, states = forward(prob, kref, s, uG, store=True, rot=rot)
    res = adjoint(prob, kref, s, uG, states, rot=rot)
    g_kref, g_s, g_uG = res[:3]
    g_kr = strip_margin(g_kref, prob.margin)
    g_gb = g_kr * kappa_ref_deriv(gb, prob.kappa_max, prob.q)
    g_gt = g_gb * projection_deriv(gt, prob.beta, prob.eta)
    g_gamma = density_filter_T(g_gt, prob.filter_R)
    g_knots = knot_gradient(prob, g_s, g_uG)
    if rot is not None:
        return J, g_gamma, g_knots, angle_gradient(prob, res[3], res[4], len(aknots))
    return J, g_gamma, g_knots
