"""Combined semi-smooth Newton / primal-dual active-set loop (oracle; test infrastructure only).

Follows the algorithm of Section 3 (printed in LaTeX comments there) for one
loading step of Formulation 1 with the irreversibility constraint
phi <= phi_old (Section 2):

  repeat for k = 0, 1, ...
    1. residual F = -r(U^k)                                   (model.gradient)
    2. active set A_k = {i : F_phi,i / m_i + c (phi_i - phi_old,i) > tau}
       with the lumped phase-field mass m (the paper's "B").  The paper gives
       neither c nor the threshold of its printed rule; both are read in units
       of the crack-energy stiffness G_c/eps, which makes the two terms of the
       indicator commensurate: c = c_rel G_c/eps, tau = tol_active G_c/eps
       (tol_active = 1e-10: indicators below it are numerically zero, e.g. far
       from the crack where they are ~1e-11 .. 1e-13); indices
       that change membership ``cycle_lock`` times in this loading step are
       locked active (Section 3: alternating active-set indices are detected
       and constrained to avoid cycles)
    3. Jacobian G (Section 3.1 blocks)
    4. eliminate Dirichlet displacement rows/cols and active phase-field
       rows/cols: active entries get delta phi_i = phi_old,i - phi_i, whose
       column contribution moves to the right-hand side
    5. solve the reduced system EXACTLY.  M_u_phi = 0, so the system is block
       lower triangular: M_uu du = F_u, then M_phi_phi dphi = F_phi - M_phi_u du
       (sparse direct solves; the paper uses GMRES + AMG for this step)
    6. line search: omega = 1, halved while the scaled reduced residual does
       not decrease (at most ``max_halvings`` times)
  until the active set is unchanged, the scaled reduced residual has dropped
  by ``tol_newton`` (or below the round-off floor ``atol_newton``; a loading
  step that starts near its solution cannot drop by 1e-10) and the last
  Newton step was below ``tol_step``.  A node whose indicator lies within
  tol_change G_c/eps of zero is a tie (it meets the complementarity
  conditions, to that band, as active and as free): its membership changes
  do not count and its row takes no part in the residual test.

After a converged loading step phi_prev <- phi_old, phi_old <- phi.  The
extrapolation phi~ (Section 2, "linear extrapolation in time") is read as
phi~ = phi_old in the first two loading steps (the initial crack field is not a
computed time level) and clamp(2 phi_old - phi_prev, 0, 1) afterwards.
Parity unpinned: the paper prints no value that fixes phi~ or the cycle rule.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe import Mesh
from .model import Params, gradient, jacobian, lumped_mass, scaling


@dataclass
class Options:
    c: float = 0.1               # active-set constant of step 2, in units of G_c / eps
    tol_newton: float = 1e-10    # scaled reduced residual, relative to iteration 0
    atol_newton: float = 1e-14   # ... or absolute (round-off floor of the scaled residual)
    tol_step: float = 1e-9       # last Newton step, relative to the iterate (per block, inf-norm)
    max_newton: int = 50
    max_halvings: int = 10
    cycle_lock: int = 3
    full_jacobian: bool = False
    tol_active: float = 1e-10    # threshold tau of step 2, in units of G_c / eps
    tol_change: float = 1e-9     # membership changes within this band (G_c/eps units) are ties
    trace: bool = False          # keep (raw set, locked set, A_k) of every iteration in the report


@dataclass
class StepReport:
    converged: bool = False
    newton_its: int = 0
    active: int = 0
    changed: int = 0
    locked: int = 0
    ties: int = 0
    linesearch_fails: int = 0
    rho0: float = 0.0
    rho: float = 0.0
    history: List[float] = field(default_factory=list)
    omegas: List[float] = field(default_factory=list)
    trace: list = field(default_factory=list)   # (raw, locked, A) per iteration when Options.trace


@dataclass
class State:
    mesh: Mesh
    prm: Params
    u: np.ndarray
    phi: np.ndarray
    phi_old: np.ndarray
    phi_prev: Optional[np.ndarray] = None
    steps_done: int = 0
    active: Optional[np.ndarray] = None
    indicator: Optional[np.ndarray] = None

    @classmethod
    def initial(cls, mesh: Mesh, prm: Params, phi0: np.ndarray):
        n = mesh.n_nodes
        return cls(mesh, prm, np.zeros((n, mesh.d)), phi0.astype(np.float64).copy(),
                   phi0.astype(np.float64).copy())

    def phi_tilde(self) -> np.ndarray:
        """Linear extrapolation in time of Section 2 (parity unpinned against the paper).

        Extrapolation needs two computed time levels: the initial crack field is
        a description of the crack, not a solution, so the first two loading
        steps use phi~ = phi_old; from step 3 on phi~ = clamp(2 phi_old -
        phi_prev, 0, 1) (uniform steps).
        """
        if self.steps_done <= 1 or self.phi_prev is None:
            return self.phi_old.copy()
        return np.clip(2.0 * self.phi_old - self.phi_prev, 0.0, 1.0)


def _reduced_scaled(F, S, free):
    return np.where(free, F / S, 0.0)


def _update(u, phi, phi_old, du, dphi, active, omega):
    u_new = u + omega * du
    phi_new = phi + omega * dphi
    if omega == 1.0:
        phi_new[active] = phi_old[active]
    return u_new, phi_new


def _solve_reduced(J, rhs, free, nu_dofs, full_jacobian, cache=None):
    """Exact solve of the reduced system on the free DoFs (step 5).

    M_uu = (g(phi~) sigma(chi_j), e(chi_i)) depends on phi~ alone, which is
    fixed within a loading step, and its free rows (all but the Dirichlet
    ones) never change; ``cache`` (one dict per loading step) keeps its sparse
    LU factors, so every Newton iteration solves with the same factors a fresh
    factorization would produce.
    """
    x = np.zeros_like(rhs)
    if full_jacobian:
        idx = np.flatnonzero(free)
        Jff = J[idx][:, idx].tocsc()
        x[idx] = spla.spsolve(Jff, rhs[idx])
        return x
    fu = np.flatnonzero(free[:nu_dofs])
    fp = np.flatnonzero(free[nu_dofs:])
    Juu = J[:nu_dofs, :nu_dofs]
    Jpu = J[nu_dofs:, :nu_dofs]
    Jpp = J[nu_dofs:, nu_dofs:]
    if fu.size:
        if cache is None:
            cache = {}
        if "uu" not in cache:
            cache["uu"] = spla.splu(Juu[fu][:, fu].tocsc())
        x[fu] = cache["uu"].solve(rhs[fu])
    rp = rhs[nu_dofs:] - Jpu @ x[:nu_dofs]
    if fp.size:
        x[nu_dofs + fp] = spla.spsolve(Jpp[fp][:, fp].tocsc(), rp[fp])
    return x


def active_threshold(prm: Params, opts: Options) -> float:
    """tau of step 2: the threshold of the printed active-set rule, tol_active G_c / eps."""
    return opts.tol_active * prm.Gc / prm.eps


def active_constant(prm: Params, opts: Options) -> float:
    """c of step 2: c_rel G_c / eps."""
    return opts.c * prm.Gc / prm.eps


def active_indicator(F_phi, m, phi, phi_old, c):
    """lambda_i + c (phi_i - phi_old,i) with lambda = F_phi / m (step 2)."""
    return F_phi / m + c * (phi - phi_old)


def loading_step(st: State, p: float, opts: Options = Options()) -> StepReport:
    """Solve one loading step with pressure p; updates ``st`` in place."""
    mesh = st.mesh
    prm = replace(st.prm, p=p)
    d, n = mesh.d, mesh.n_nodes
    nu_dofs = d * n
    phit = st.phi_tilde()
    S = scaling(mesh, prm, phit)
    m = lumped_mass(mesh)
    fixed_u = np.repeat(mesh.boundary_nodes(), d)
    u, phi, phi_old = st.u.copy(), st.phi.copy(), st.phi_old
    rep = StepReport()
    raw_prev = A_prev = None
    toggles = np.zeros(n, dtype=np.int64)
    locked = np.zeros(n, dtype=bool)
    last_small = False
    lu_cache = {}          # factors of the free M_uu rows, valid for this loading step
    for k in range(opts.max_newton + 1):
        r_u, r_phi = gradient(mesh, prm, u, phi, phit)
        F = -np.concatenate([r_u.ravel(), r_phi])
        ind = active_indicator(F[nu_dofs:], m, phi, phi_old, active_constant(prm, opts))
        raw = ind > active_threshold(prm, opts)
        if raw_prev is not None:
            toggles += raw != raw_prev
            locked |= toggles >= opts.cycle_lock
        A = raw | locked
        if opts.trace:
            rep.trace.append((raw.copy(), locked.copy(), A.copy()))
        free = ~np.concatenate([fixed_u, A])
        rho = _reduced_scaled(F, S, free)
        rho_inf = float(np.max(np.abs(rho))) if rho.size else 0.0
        if k == 0:
            rep.rho0 = rho_inf
        rep.history.append(rho_inf)
        rep.changed = int(np.count_nonzero(A != A_prev)) if A_prev is not None else int(A.sum())
        band = opts.tol_change * prm.Gc / prm.eps
        tie = np.abs(ind) <= band
        unchanged = A_prev is not None and not np.any((A != A_prev) & ~tie)
        # a tie row meets complementarity as either member: it takes no part in the test
        rho_stop = rho.copy()
        rho_stop[nu_dofs:][tie] = 0.0
        rho_stop_inf = float(np.max(np.abs(rho_stop))) if rho.size else 0.0
        done = (unchanged
                and rho_stop_inf <= max(opts.tol_newton * rep.rho0, opts.atol_newton)
                and last_small) or rep.rho0 == 0.0
        if done or k == opts.max_newton:
            rep.converged = bool(done)
            rep.newton_its = k
            rep.rho = rho_inf
            st.active, st.indicator = A, ind
            break
        J = jacobian(mesh, prm, u, phi, phit, full_jacobian=opts.full_jacobian)
        dUA = np.zeros(nu_dofs + n)
        dUA[nu_dofs:][A] = phi_old[A] - phi[A]
        rhs = F - J @ dUA
        dU = dUA + _solve_reduced(J, rhs, free, nu_dofs, opts.full_jacobian, lu_cache)
        du, dphi = dU[:nu_dofs].reshape(n, d), dU[nu_dofs:]
        u1, phi1 = _update(u, phi, phi_old, du, dphi, A, 1.0)
        small = (np.max(np.abs(du), initial=0.0) <= opts.tol_step * np.max(np.abs(u1), initial=0.0)
                 and np.max(np.abs(dphi), initial=0.0) <= opts.tol_step * np.max(np.abs(phi1), initial=0.0))
        omega = 1.0
        if not small:
            r_old = float(np.linalg.norm(rho))
            for t in range(opts.max_halvings + 1):
                ut, pt = _update(u, phi, phi_old, du, dphi, A, omega)
                gu, gp = gradient(mesh, prm, ut, pt, phit)
                Ft = -np.concatenate([gu.ravel(), gp])
                if float(np.linalg.norm(_reduced_scaled(Ft, S, free))) < r_old:
                    break
                if t == opts.max_halvings:
                    omega = 1.0
                    rep.linesearch_fails += 1
                    break
                omega *= 0.5
        rep.omegas.append(omega)
        u, phi = _update(u, phi, phi_old, du, dphi, A, omega)
        last_small = small
        raw_prev, A_prev = raw, A
    rep.active = int(A.sum())
    rep.locked = int(locked.sum())
    rep.ties = int(np.count_nonzero(np.abs(ind) <= active_threshold(prm, opts)))
    st.u, st.phi = u, phi
    st.phi_prev, st.phi_old = st.phi_old, phi.copy()
    st.steps_done += 1
    return rep


def solve_loading_steps(st: State, pressures, opts: Options = Options()) -> List[StepReport]:
    """Formulation 1 for loading steps n = 1, 2, ... with the given pressures."""
    return [loading_step(st, p, opts) for p in pressures]
