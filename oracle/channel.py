"""One RK3 / Crank-Nicolson step of the channel flow, written out plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is computed (paper Sec. 3.1 and Sec. 3.2, and the readings stated below)
----------------------------------------------------------------------------
Incompressible Navier-Stokes in a plane channel ``y in [-1, 1]`` (half height
1, bulk velocity 1, ``nu = 1 / Re_b``) in rotational form,
``du/dt = H - grad p + nu lap u + f_x e_x`` with ``H = u x omega``.  The state
is the wall-normal velocity ``v`` and vorticity ``g = omega_y`` per Fourier
mode, plus the mean profiles ``U(y)``, ``W(y)``, all as Chebyshev
coefficients (Sec. 3.1: Fourier in x, z; Chebyshev in y).

Per mode ``k != 0`` (``k^2 = kx^2 + kz^2``)::

    d(lap v)/dt = h_v + nu lap lap v ,  h_v = -k^2 H_y - D(i kx H_x + i kz H_z)
    d g / dt    = h_g + nu lap g ,      h_g = i kz H_x - i kx H_z

Mean mode: ``dU/dt = <H_x> + nu D^2 U + f_x`` with ``f_x`` set every stage so
that the flow rate ``int U dy = 2`` stays constant; ``dW/dt = <H_z> + nu D^2 W``.

Time scheme (Sec. 3.1: Crank-Nicolson for the linear terms, third-order
Runge-Kutta for the nonlinear terms), low-storage form, stage k = 1..3::

    q_k - beta_k dt L q_k = q_{k-1} + alpha_k dt L q_{k-1}
                            + dt (gamma_k N_{k-1} + zeta_k N_{k-2})
    gamma = (8/15, 5/12, 3/4), zeta = (0, -17/60, -5/12),
    alpha_k = beta_k = (gamma_k + zeta_k) / 2.

The nonlinear term is evaluated with the 3/2 rule: velocity and vorticity are
taken to the ``3nx/2 x 3nz/2`` grid at every Chebyshev node, multiplied, and
truncated back.  Wall-normal problems are Chebyshev-tau: the equation holds
for coefficients ``0..N-2`` and two boundary rows close each system.  The
fourth-order ``v`` problem is solved here as ONE coupled dense system for the
unknowns ``(phi, v)``, ``phi = lap v``: tau rows of
``(D^2 - lambda) phi = r``, tau rows of ``(D^2 - k^2) v = phi`` and the four
wall conditions ``v(+1) = 0, v(-1) = v_w, Dv(+1) = Dv(-1) = 0``.  (The CUDA
path reaches the same solution through an influence-matrix superposition.)
The mean profile is one dense system with the unknown forcing ``f_x`` and the
flow-rate row appended.

Open channel (``top_bc = 1``; Sec. 3.1: an open channel of height h with a
free-slip top): ``y in [-1, 1]`` is the whole channel, so Re_b and Re_tau
are based on the height 2 (``nu = 2 / Re_b``, ``y+ = (1 + y) Re_tau / 2``),
and the top rows become ``Dg(+1) = 0``, ``D^2 v(+1) = 0`` (with ``v(+1) = 0``),
``DU(+1) = DW(+1) = 0``.

Wall action (Sec. 3.2): clipped to ``[-u_tau, u_tau]``, plane mean removed
(zero net mass flux, Sec. 4.1), ramped linearly from the previous action over
the actuation interval; stage k of step s sees the ramp at its end time.
Opposition control (Sec. 4.1 equation): ``v_w = -alpha (v(y_s) - <v(y_s)>)``.
Observation (Sec. 3.2): u and v on the wall-parallel plane at the first
Chebyshev node with ``y+ >= y_sense_plus`` above the lower wall.  Reward
(Sec. 3.2): ``1 - tau_w / tau_ref`` with ``tau_w`` the wall shear of the lower
wall averaged over the steps of one action.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import spectral as sp

# Low-storage RK3 coefficients (third-order RK for the nonlinear term).
GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)
ALPHA = tuple((g + z) / 2.0 for g, z in zip(GAMMA, ZETA))
BETA = ALPHA
# Fraction of the step reached at the end of each stage: 8/15, 2/3, 1.
C_END = (8.0 / 15.0, 2.0 / 3.0, 1.0)


@dataclass
class Params:
    nx: int
    ny: int
    nz: int
    lx: float
    lz: float
    re_tau: float = 180.0
    re_bulk: float = 2800.0
    dt: float = 0.005
    steps_per_action: int = 1
    y_sense_plus: float = 15.0
    control: int = 0          # 0 external action, 1 opposition control
    alpha: float = 1.0        # opposition gain
    tau_ref: float = 0.0      # 0 -> (Re_tau / Re_b)^2
    top_bc: int = 0           # 0 no-slip wall at y = +1, 1 free slip (open channel)

    @property
    def height(self) -> float:
        """Length on which Re_b and Re_tau are based, in units of y: the
        half-height 1 of the closed channel; the whole height 2 of the open
        channel (Sec. 3.1: an open channel of height h)."""
        return 2.0 if self.top_bc == 1 else 1.0

    @property
    def nu(self) -> float:
        return self.height / self.re_bulk

    @property
    def u_tau(self) -> float:
        return self.re_tau / self.re_bulk

    @property
    def tau_reference(self) -> float:
        return self.tau_ref if self.tau_ref > 0 else self.u_tau ** 2


def sensing_node(N: int, re_tau: float, y_plus: float, height: float = 1.0) -> int:
    """First Gauss-Lobatto node, walking up from the lower wall, with y+ >= y_plus.

    Sec. 3.2: the sampling height is rounded up to a Chebyshev node;
    y+ = (1 + y) u_tau / nu = (1 + y) Re_tau / height measured from the lower
    wall (height: the length Re_tau is based on, in units of y).
    """
    for j in range(N, -1, -1):
        yj = math.cos(math.pi * j / N)
        if (1.0 + yj) * re_tau / height >= y_plus:
            return j
    return 0


class Operators:
    """Dense operators of one grid."""

    def __init__(self, p: Params):
        self.p = p
        N = p.ny - 1
        self.N = N
        self.D = sp.cheb_diff(N)
        self.D2 = self.D @ self.D
        self.S = sp.cheb_synthesis(N)
        self.A = sp.cheb_analysis(N)
        self.Tp = sp.cheb_at_plus1(N)
        self.Tm = sp.cheb_at_minus1(N)
        self.dTp = self.Tp @ self.D      # T_n'(+1)
        self.dTm = self.Tm @ self.D      # T_n'(-1)
        self.d2Tp = self.Tp @ self.D2    # T_n''(+1)
        self.free_slip = p.top_bc == 1
        self.wint = sp.cheb_integral(N)
        kx, kz, kept = sp.wavenumbers(p.nx, p.nz, p.lx, p.lz)
        self.kx = kx[None, :, None]          # [1, nxh, 1]
        self.kz = kz[:, None, None]          # [nz, 1, 1]
        self.kept = kept
        self.k2 = self.kx ** 2 + self.kz ** 2
        self.mx = 3 * p.nx // 2
        self.mz = 3 * p.nz // 2
        self.js = sensing_node(N, p.re_tau, p.y_sense_plus, p.height)

    # coefficient-space derivative along the last axis
    def d(self, a):
        return a @ self.D.T

    def d2(self, a):
        return a @ self.D2.T


# --------------------------------------------------------------------------
# state helpers (canonical layout [ny][nz][nx/2] <-> pencils [nz][nx/2][ny])
# --------------------------------------------------------------------------

def to_pencils(a):
    return np.ascontiguousarray(np.moveaxis(a, 0, -1))


def from_pencils(a):
    return np.ascontiguousarray(np.moveaxis(a, -1, 0))


def new_state(fields: dict, p: Params) -> dict:
    """Oracle state from a seeded field dict (v, g, U, W in the canonical layout)."""
    nxh = p.nx // 2
    return {
        "v": to_pencils(np.asarray(fields["v"], np.complex128)),
        "g": to_pencils(np.asarray(fields["g"], np.complex128)),
        "U": np.asarray(fields["U"], np.float64).copy(),
        "W": np.asarray(fields["W"], np.float64).copy(),
        "vw": np.zeros((p.nz, nxh), np.complex128),
        "t": 0.0,
        "steps": 0,
    }


# --------------------------------------------------------------------------
# velocity and vorticity from (v, g, U, W)
# --------------------------------------------------------------------------

def velocity_vorticity(st: dict, ops: Operators) -> dict:
    """Coefficients of u, v, w, omega_x, omega_y, omega_z for every mode.

    Continuity ``i kx u + Dv + i kz w = 0`` and ``g = i kz u - i kx w`` give
    ``u = (i kx Dv - i kz g) / k^2``, ``w = (i kz Dv + i kx g) / k^2``; the
    curl gives ``omega_x = Dw - i kz v``, ``omega_z = i kx v - Du``.  The mean
    mode carries ``u = U``, ``w = W``, ``omega_x = DW``, ``omega_z = -DU``.
    """
    v, g = st["v"], st["g"]
    kx, kz, k2 = ops.kx, ops.kz, ops.k2
    k2s = np.where(k2 == 0.0, 1.0, k2)
    dv = ops.d(v)
    d2v = ops.d(dv)
    dg = ops.d(g)
    u = (1j * kx * dv - 1j * kz * g) / k2s
    w = (1j * kz * dv + 1j * kx * g) / k2s
    du = (1j * kx * d2v - 1j * kz * dg) / k2s
    dw = (1j * kz * d2v + 1j * kx * dg) / k2s
    ox = dw - 1j * kz * v
    oz = 1j * kx * v - du
    oy = g.copy()
    vv = v.copy()
    U, W = st["U"], st["W"]
    u[0, 0] = U
    w[0, 0] = W
    vv[0, 0] = 0.0
    ox[0, 0] = ops.D @ W
    oy[0, 0] = 0.0
    oz[0, 0] = -(ops.D @ U)
    out = {"u": u, "v": vv, "w": w, "ox": ox, "oy": oy, "oz": oz}
    for f in out.values():
        f[~ops.kept] = 0.0
    return out


def nonlinear(st: dict, ops: Operators):
    """Dealiased ``H = u x omega`` and the right-hand sides h_v, h_g.

    Returns ``(hv, hg, Hx00, Hz00, H)``: pencils of h_v and h_g, the mean-mode
    coefficients of H_x and H_z (real parts), and the three H coefficient
    fields.
    """
    f = velocity_vorticity(st, ops)
    # coefficients -> node values (last axis), then [node][nz][nxh]
    nodes = {k: from_pencils(f[k] @ ops.S.T) for k in NODE_FIELDS}
    Hn = nonlinear_nodes(nodes, ops)
    H = {c: to_pencils(Hn[c]) @ ops.A.T for c in "xyz"}   # Chebyshev coefficients
    hv, hg, Hx00, Hz00 = assemble(H, ops)
    return hv, hg, Hx00, Hz00, H


NODE_FIELDS = ("u", "v", "w", "ox", "oy", "oz")


def nonlinear_nodes(nodes: dict, ops: Operators) -> dict:
    """3/2-dealiased ``H = u x omega`` plane by plane.

    ``nodes[name]``: ``[ny][nz][nx/2]`` Fourier coefficients at each node of
    u, v, w, omega_x, omega_y, omega_z.  Returns the kept Fourier
    coefficients of H_x, H_y, H_z at each node (same layout).
    """
    p = ops.p
    phys = {k: sp.to_physical(nodes[k], p.nx, p.nz, ops.mx, ops.mz) for k in NODE_FIELDS}
    u, v, w = phys["u"], phys["v"], phys["w"]
    ox, oy, oz = phys["ox"], phys["oy"], phys["oz"]
    Hphys = {
        "x": v * oz - w * oy,
        "y": w * ox - u * oz,
        "z": u * oy - v * ox,
    }
    return {c: sp.to_spectral(Hphys[c], p.nx, p.nz, ops.mx, ops.mz) for c in "xyz"}


def assemble(H: dict, ops: Operators):
    """Right-hand sides of the v and g equations from the coefficients of H.

    ``h_v = -k^2 H_y - D(i kx H_x + i kz H_z)`` (y component of
    ``-curl curl H``), ``h_g = i kz H_x - i kx H_z`` (y component of
    ``curl H``); the mean mode returns the real parts of ``H_x`` and ``H_z``.
    """
    kx, kz, k2 = ops.kx, ops.kz, ops.k2
    hv = -k2 * H["y"] - ops.d(1j * kx * H["x"] + 1j * kz * H["z"])
    hg = 1j * kz * H["x"] - 1j * kx * H["z"]
    hv[0, 0] = 0.0
    hg[0, 0] = 0.0
    hv[~ops.kept] = 0.0
    hg[~ops.kept] = 0.0
    Hx00 = np.real(H["x"][0, 0]).copy()
    Hz00 = np.real(H["z"][0, 0]).copy()
    return hv, hg, Hx00, Hz00


# --------------------------------------------------------------------------
# dense Chebyshev-tau systems
# --------------------------------------------------------------------------

def _solve_real(M, rhs):
    """Solve real systems M x = rhs for complex rhs (real and imaginary parts)."""
    b = np.stack([rhs.real, rhs.imag], axis=-1)
    x = np.linalg.solve(M, b)
    return x[..., 0] + 1j * x[..., 1]


# The dense systems of independent pencils are assembled and solved in chunks
# of at most PENCIL_CHUNK pencils, so that the stacked (P, n, n) matrices of a
# large grid (32768 pencils of 386 x 386 at 256 x 193 x 256) never exist at
# once.  Each pencil's system and its LU solve are the same as in one batch.
# The chunks are independent; `_pencil_starmap(func, tasks)` runs them
# (serially by default; a caller may install a process pool's starmap with
# set_pencil_starmap).
PENCIL_CHUNK = 256


def _serial_starmap(func, tasks):
    return [func(*t) for t in tasks]


_pencil_starmap = _serial_starmap


def set_pencil_starmap(fn=None):
    """Run the pencil chunks with ``fn(func, list_of_argument_tuples)``
    (serially in this process if None)."""
    global _pencil_starmap
    _pencil_starmap = _serial_starmap if fn is None else fn


def _chunked(func, fixed: tuple, *per_pencil):
    """``func(*fixed, *chunk)`` over chunks of the per-pencil arrays, concatenated."""
    P = per_pencil[0].shape[0]
    if P == 0:
        return func(*fixed, *per_pencil)
    tasks = [fixed + tuple(a[i:i + PENCIL_CHUNK] for a in per_pencil) for i in range(0, P, PENCIL_CHUNK)]
    return np.concatenate(_pencil_starmap(func, tasks), axis=0)


def tau_dirichlet(ops: Operators, lam: np.ndarray, r: np.ndarray,
                  top: np.ndarray, bottom: np.ndarray, top_neumann: bool = False) -> np.ndarray:
    """Solve ``(D^2 - lam) f = r`` (tau rows 0..N-2), ``f(+1) = top``, ``f(-1) = bottom``.

    ``lam[P]``, ``r[P, N+1]`` (complex), ``top/bottom[P]`` -> ``f[P, N+1]``.
    With ``top_neumann`` the top row is ``Df(+1) = top`` (free slip).
    """
    top_row = ops.dTp if top_neumann else ops.Tp
    return _chunked(_tau_dirichlet_pencils, (ops.D2, top_row, ops.Tm), lam, r, top, bottom)


def _tau_dirichlet_pencils(D2, top_row, bot_row, lam, r, top, bottom):
    """Dense tau systems of ``tau_dirichlet`` for one set of pencils."""
    N = D2.shape[0] - 1
    P = lam.shape[0]
    M = np.zeros((P, N + 1, N + 1))
    M[:, : N - 1, :] = D2[None, : N - 1, :]
    idx = np.arange(N - 1)
    M[:, idx, idx] -= lam[:, None]
    M[:, N - 1, :] = top_row
    M[:, N, :] = bot_row
    b = np.zeros((P, N + 1), np.complex128)
    b[:, : N - 1] = r[:, : N - 1]
    b[:, N - 1] = top
    b[:, N] = bottom
    return _solve_real(M, b)


def coupled_v(ops: Operators, lam: np.ndarray, k2: np.ndarray, r: np.ndarray,
              vw: np.ndarray) -> np.ndarray:
    """The v problem as one dense system in the unknowns (phi, v).

    Rows: tau rows of ``(D^2 - lam) phi = r``; tau rows of
    ``(D^2 - k^2) v - phi = 0``; ``v(+1) = 0``, ``v(-1) = vw``,
    ``Dv(+1) = 0``, ``Dv(-1) = 0``.  Returns v coefficients ``[P, N+1]``.
    Free-slip top (``ops.free_slip``): ``D^2 v(+1) = 0`` replaces
    ``Dv(+1) = 0`` (u, w free of shear there, and by continuity
    ``D^2 v = -(i kx Du + i kz Dw) = 0``).
    """
    third = ops.d2Tp if ops.free_slip else ops.dTp
    return _chunked(_coupled_v_pencils, (ops.D2, ops.Tp, ops.Tm, third, ops.dTm), lam, k2, r, vw)


def _coupled_v_pencils(D2, Tp, Tm, third, dTm, lam, k2, r, vw):
    """Dense coupled (phi, v) systems of ``coupled_v`` for one set of pencils."""
    N = D2.shape[0] - 1
    n1 = N + 1
    P = lam.shape[0]
    M = np.zeros((P, 2 * n1, 2 * n1))
    idx = np.arange(N - 1)
    # (D^2 - lam) phi = r
    M[:, : N - 1, :n1] = D2[None, : N - 1, :]
    M[:, idx, idx] -= lam[:, None]
    # (D^2 - k^2) v - phi = 0
    M[:, N - 1 + idx, idx] = -1.0
    M[:, N - 1: 2 * N - 2, n1:] = D2[None, : N - 1, :]
    M[:, N - 1 + idx, n1 + idx] -= k2[:, None]
    # wall rows
    M[:, 2 * N - 2, n1:] = Tp
    M[:, 2 * N - 1, n1:] = Tm
    M[:, 2 * N, n1:] = third
    M[:, 2 * N + 1, n1:] = dTm
    b = np.zeros((P, 2 * n1), np.complex128)
    b[:, : N - 1] = r[:, : N - 1]
    b[:, 2 * N - 1] = vw
    x = _solve_real(M, b)
    return x[:, n1:]


def mean_cfr(ops: Operators, lam0: float, cforce: float, r: np.ndarray,
             flux: float = 2.0):
    """Mean streamwise profile at constant flow rate.

    Unknowns ``(U, f)``: tau rows of ``(D^2 - lam0) U + cforce f T_0 = r``,
    ``U(+1) = U(-1) = 0`` and ``int_{-1}^{1} U dy = flux``.  Free-slip top:
    ``DU(+1) = 0`` replaces ``U(+1) = 0``.
    Returns ``(U, f)``.
    """
    N = ops.N
    n1 = N + 1
    M = np.zeros((n1 + 1, n1 + 1))
    M[: N - 1, :n1] = ops.D2[: N - 1, :]
    M[np.arange(N - 1), np.arange(N - 1)] -= lam0
    M[0, n1] = cforce
    M[N - 1, :n1] = ops.dTp if ops.free_slip else ops.Tp
    M[N, :n1] = ops.Tm
    M[N + 1, :n1] = ops.wint
    b = np.zeros(n1 + 1)
    b[: N - 1] = r[: N - 1]
    b[N + 1] = flux
    x = np.linalg.solve(M, b)
    return x[:n1], x[n1]


def mean_dirichlet(ops: Operators, lam0: float, r: np.ndarray) -> np.ndarray:
    """Mean spanwise profile: tau rows of ``(D^2 - lam0) W = r``, ``W(+-1) = 0``
    (``DW(+1) = 0`` under a free-slip top)."""
    N = ops.N
    M = np.zeros((N + 1, N + 1))
    M[: N - 1] = ops.D2[: N - 1]
    M[np.arange(N - 1), np.arange(N - 1)] -= lam0
    M[N - 1] = ops.dTp if ops.free_slip else ops.Tp
    M[N] = ops.Tm
    b = np.zeros(N + 1)
    b[: N - 1] = r[: N - 1]
    return np.linalg.solve(M, b)


# --------------------------------------------------------------------------
# one RK3 stage / step
# --------------------------------------------------------------------------

def stage(st: dict, ops: Operators, k: int, vw: np.ndarray, prev: dict | None) -> dict:
    """Advance ``st`` in place through RK3 stage ``k`` (0-based); return this stage's N terms."""
    p = ops.p
    nu, dt = p.nu, p.dt
    a, b, gm, ze = ALPHA[k], BETA[k], GAMMA[k], ZETA[k]
    hv, hg, Hx00, Hz00, _ = nonlinear(st, ops)
    if prev is None:
        prev = {"hv": np.zeros_like(hv), "hg": np.zeros_like(hg),
                "Hx00": np.zeros_like(Hx00), "Hz00": np.zeros_like(Hz00)}
    bdn = b * dt * nu
    v, g = st["v"], st["g"]
    k2 = ops.k2
    # active pencils: kept rows, not the mean
    act = np.broadcast_to(ops.kept[:, None], k2.shape[:2]).copy()
    act[0, 0] = False
    lam_full = (k2[..., 0] + 1.0 / bdn)

    # wall-normal vorticity
    lap_g = ops.d2(g) - k2 * g
    rg = -(g + a * dt * nu * lap_g + dt * (gm * hg + ze * prev["hg"])) / bdn
    # wall-normal velocity (phi = lap v)
    phi = ops.d2(v) - k2 * v
    lap_phi = ops.d2(phi) - k2 * phi
    rphi = -(phi + a * dt * nu * lap_phi + dt * (gm * hv + ze * prev["hv"])) / bdn

    lam = lam_full[act]
    zero = np.zeros(lam.shape[0])
    g_new = np.zeros_like(g)
    v_new = np.zeros_like(v)
    g_new[act] = tau_dirichlet(ops, lam, rg[act], zero, zero, top_neumann=ops.free_slip)
    v_new[act] = coupled_v(ops, lam, k2[..., 0][act], rphi[act], vw[act])

    # mean flow
    lam0 = 1.0 / bdn
    U, W = st["U"], st["W"]
    rU = -(U + a * dt * nu * (ops.D2 @ U) + dt * (gm * Hx00 + ze * prev["Hx00"])) / bdn
    rW = -(W + a * dt * nu * (ops.D2 @ W) + dt * (gm * Hz00 + ze * prev["Hz00"])) / bdn
    U_new, fx = mean_cfr(ops, lam0, (a + b) / (b * nu), rU)
    W_new = mean_dirichlet(ops, lam0, rW)

    st["v"], st["g"], st["U"], st["W"] = v_new, g_new, U_new, W_new
    st["fx"] = fx
    return {"hv": hv, "hg": hg, "Hx00": Hx00, "Hz00": Hz00}


def wall_shear(U: np.ndarray, ops: Operators) -> float:
    """tau_w = nu dU/dy at the lower wall y = -1 (wall-averaged shear, Sec. 3.2)."""
    return ops.p.nu * float(ops.dTm @ U)


def rk3_step(st: dict, ops: Operators, vw_old: np.ndarray, vw_new: np.ndarray,
             s: int) -> float:
    """One full RK3 step (three stages); step ``s`` of the current action.

    Stage k applies the wall velocity ``vw_old + theta (vw_new - vw_old)``
    with ``theta = (s + c_k) / steps_per_action`` (linear ramp over the
    actuation interval, Sec. 3.2).  Returns tau_w after the step.
    """
    prev = None
    for k in range(3):
        theta = (s + C_END[k]) / ops.p.steps_per_action
        vw = vw_old + theta * (vw_new - vw_old)
        prev = stage(st, ops, k, vw, prev)
    st["t"] += ops.p.dt
    st["steps"] += 1
    return wall_shear(st["U"], ops)


# --------------------------------------------------------------------------
# environment step: action, evolve, observe, reward
# --------------------------------------------------------------------------

def action_spectrum(action: np.ndarray, ops: Operators) -> np.ndarray:
    """Wall action ``[nz][nx]`` -> kept Fourier modes of the wall velocity.

    Clip to ``[-u_tau, u_tau]`` (Sec. 3.2), then remove the plane mean (zero
    net mass flux); the mean mode is set to zero and Nyquist content dropped.
    """
    p = ops.p
    a = np.clip(np.asarray(action, np.float64), -p.u_tau, p.u_tau)
    a = a - a.mean()
    F = sp.to_spectral(a, p.nx, p.nz, p.nx, p.nz)
    F[0, 0] = 0.0
    return F


def plane_at_node(coef: np.ndarray, ops: Operators, j: int) -> np.ndarray:
    """Fourier coefficients of a field at Gauss-Lobatto node j (``[nz][nxh]``)."""
    return coef @ ops.S[j]


def opposition_spectrum(st: dict, ops: Operators) -> np.ndarray:
    """Sec. 4.1: v_w = -alpha (v(y_s) - <v(y_s)>), spectrally: every mode but the mean."""
    F = -ops.p.alpha * plane_at_node(st["v"], ops, ops.js)
    F[0, 0] = 0.0
    return F


def observation(st: dict, ops: Operators) -> np.ndarray:
    """u and v on the sensing plane, physical ``[2][nz][nx]`` (Sec. 3.2)."""
    p = ops.p
    f = velocity_vorticity(st, ops)
    us = plane_at_node(f["u"], ops, ops.js)
    vs = plane_at_node(f["v"], ops, ops.js)
    return np.stack([sp.to_physical(us, p.nx, p.nz, p.nx, p.nz),
                     sp.to_physical(vs, p.nx, p.nz, p.nx, p.nz)])


def env_step(st: dict, ops: Operators, action: np.ndarray | None = None):
    """One interaction: set the action, evolve ``steps_per_action`` steps, observe.

    Returns ``(obs, tau_w_mean, reward)``.
    """
    p = ops.p
    if p.control == 1:
        vw_new = opposition_spectrum(st, ops)
    else:
        vw_new = action_spectrum(action, ops)
    vw_old = st["vw"]
    taus = [rk3_step(st, ops, vw_old, vw_new, s) for s in range(p.steps_per_action)]
    st["vw"] = vw_new
    tau = float(np.mean(taus))
    reward = 1.0 - tau / p.tau_reference
    return observation(st, ops), tau, reward


def canonical(st: dict) -> dict:
    """State in the canonical (library) layout."""
    return {"v": from_pencils(st["v"]), "g": from_pencils(st["g"]),
            "U": st["U"].copy(), "W": st["W"].copy(), "vw": st["vw"].copy(),
            "t": st["t"], "steps": st["steps"]}
