"""FP64 oracle of the SCH discretisation (test infrastructure only).

Follows Sec. 2 of the paper:

* periodic P1 (continuous piecewise-linear) space V_h on n uniform cells of
  width h = L / n, nodes x_i = i h (indices mod n);
* the Helmholtz relation, Eq. sde1 first line:
  (u, psi) + alpha^2 (u_x, psi_x) = (m, psi)  ->  (M + alpha^2 K) u = M m;
* the implicit-midpoint step, Eq. fde1:
  (m1 - m0, phi) + mu dt (mbar_x, phi_x) + (mbar dv_x, phi) - (mbar dv, phi_x) = 0
  with mbar = (m0 + m1) / 2 and dv = dt (u0 + u1) / 2 + dU  (the increment
  Delta v^{n+1/2} of the text under Eq. fde1);
* SALT noise, either the mode expansion named in Sec. 2, dU = sum_k xi_k dW^k
  with the mode functions interpolated at the nodes, plus the nudging drift of
  Sec. 3.1.3: dU_i = sum_k xi_k(x_i) (dW_k + lambda_k dt); or the paper's
  Matern field (Eq. noise_solve, Eq. noise_solve2): one Brownian motion per
  cell, dW_h = sum_c h^{-1/2} 1_c dW_c in DG0, and k chained P1 solves
  (U_j, v) + kappa^{-2} (U_j', v') = eta (dW_h, v) for j = 1, (U_{j-1}, v)
  after, dU = U_k; the drift lambda is a DG0 field added to dW.

Every matrix is assembled element by element from exact integrals of products
of linear functions on the reference element (no quadrature), and kept as a
cyclic tridiagonal triple (a, b, c): row i reads a_i x_{i-1} + b_i x_i +
c_i x_{i+1}.  Cyclic systems are solved by Sherman-Morrison on top of LAPACK's
banded solver (scipy.linalg.solve_banded), the textbook route.

The nonlinear step (the paper names no solver) is solved by a Picard
iteration, stopped when max|m^{p+1} - m^p| <= tol max(1, max|m^{p+1}|).  Two
iterations with the same fixed point (the solution of Eq. fde1, which
``residual_quadrature`` checks independently with 3-point Gauss quadrature):

* ``scheme="li"`` (linearly implicit): with dv frozen at iterate p, solve
  (M + mu dt/2 K + 1/2 A_dv) m^{p+1} = (M - mu dt/2 K - 1/2 A_dv) m0;
* ``scheme="ea"`` (explicit advection): with mbar and dv both taken at
  iterate p, solve (M + mu dt/2 K) m^{p+1} = (M - mu dt/2 K) m0 - A(mbar^p, dv^p),
  a constant matrix, at the price of a slower contraction;

and in both u^{p+1} = H^{-1} M m^{p+1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_banded

# exact integrals of N_a N_b over the reference element [0, 1]
_MLOC = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
# d N_a / d xi for N_0 = 1 - xi, N_1 = xi
_DN = np.array([-1.0, 1.0])


@dataclass
class Model:
    """Parameters of the discretised SCH model."""
    L: float
    n: int
    alpha: float
    mu: float
    dt: float
    amps: np.ndarray      # a_j, j = 1..K/2
    tol: float = 1e-13
    max_iter: int = 100
    scheme: str = "li"
    noise_model: str = "modes"   # "modes" or "matern"
    kappa: float = 1.0           # Matern length scale 1 / kappa (Eq. noise_solve)
    eta: float = 1.0
    matern_k: int = 3

    @classmethod
    def from_config(cls, cfg, tol=None, max_iter=None, scheme="li") -> "Model":
        from workloads import mode_amplitudes
        return cls(L=cfg.L, n=cfg.n, alpha=cfg.alpha, mu=cfg.mu, dt=cfg.dt,
                   amps=mode_amplitudes(cfg), tol=1e-13 if tol is None else tol,
                   max_iter=100 if max_iter is None else max_iter, scheme=scheme,
                   noise_model=cfg.noise, kappa=cfg.kappa, eta=cfg.eta, matern_k=cfg.matern_k)

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def K(self) -> int:
        return 2 * len(self.amps)

    @property
    def Q(self) -> int:
        """Brownian motions per step: K for the mode expansion, one per cell for the Matern field."""
        return self.n if self.noise_model == "matern" else self.K

    @property
    def x(self) -> np.ndarray:
        return np.arange(self.n) * self.h

    # ------------------------------------------------------------------ #
    # assembly
    # ------------------------------------------------------------------ #
    def assemble(self, local: np.ndarray):
        """Cyclic tridiagonal (a, b, c) from per-element 2x2 matrices.

        ``local[e, r, s]`` couples test function of local node r with trial
        function of local node s on element e = [x_e, x_{e+1}].  Node i is local
        node 1 of element i-1 and local node 0 of element i.
        """
        prev = np.roll(local, 1, axis=0)   # element i-1 for row i
        a = prev[:, 1, 0]
        b = prev[:, 1, 1] + local[:, 0, 0]
        c = local[:, 0, 1]
        return a.copy(), b.copy(), c.copy()

    def mass(self):
        h = self.h
        return self.assemble(np.broadcast_to(h * _MLOC, (self.n, 2, 2)))

    def stiffness(self):
        h = self.h
        loc = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
        return self.assemble(np.broadcast_to(loc, (self.n, 2, 2)))

    def advection(self, v: np.ndarray):
        """Operator m -> A(m, v) with A(m, v)_i = (m v_x, phi_i) - (m v, d_x phi_i).

        On element e with local values v_0 = v_e, v_1 = v_{e+1}:
        int N_s v_x N_r dx = (v_1 - v_0) Mloc[r, s] and
        int N_s v d_x N_r dx = dN_r (Mloc[s, 0] v_0 + Mloc[s, 1] v_1).
        """
        v0 = v
        v1 = np.roll(v, -1)
        loc = np.empty((self.n, 2, 2))
        for r in range(2):
            for s in range(2):
                loc[:, r, s] = (v1 - v0) * _MLOC[r, s] - _DN[r] * (_MLOC[s, 0] * v0 + _MLOC[s, 1] * v1)
        return self.assemble(loc)

    # ------------------------------------------------------------------ #
    # cyclic tridiagonal algebra
    # ------------------------------------------------------------------ #
    @staticmethod
    def apply(tri, x: np.ndarray) -> np.ndarray:
        a, b, c = tri
        return a * np.roll(x, 1) + b * x + c * np.roll(x, -1)

    @staticmethod
    def dense(tri) -> np.ndarray:
        a, b, c = tri
        n = len(b)
        A = np.zeros((n, n))
        for i in range(n):
            A[i, (i - 1) % n] += a[i]
            A[i, i] += b[i]
            A[i, (i + 1) % n] += c[i]
        return A

    @staticmethod
    def solve(tri, d: np.ndarray) -> np.ndarray:
        """Solve the cyclic tridiagonal system by Sherman-Morrison.

        Write the matrix as T + w z^T with T tridiagonal (non-cyclic):
        gamma = -b_0, T_00 = b_0 - gamma, T_{n-1,n-1} = b_{n-1} - a_0 c_{n-1} / gamma,
        w = (gamma, 0, .., 0, c_{n-1}), z = (1, 0, .., 0, a_0 / gamma).
        """
        a, b, c = (np.asarray(t, dtype=np.float64) for t in tri)
        n = len(b)
        gamma = -b[0]
        bb = b.copy()
        bb[0] = b[0] - gamma
        bb[-1] = b[-1] - a[0] * c[-1] / gamma
        ab = np.zeros((3, n))
        ab[0, 1:] = c[:-1]
        ab[1, :] = bb
        ab[2, :-1] = a[1:]
        w = np.zeros(n)
        w[0] = gamma
        w[-1] = c[-1]
        rhs = np.stack([d, w], axis=1)
        sol = solve_banded((1, 1), ab, rhs)
        y, q = sol[:, 0], sol[:, 1]
        zy = y[0] + a[0] / gamma * y[-1]
        zq = q[0] + a[0] / gamma * q[-1]
        return y - (zy / (1.0 + zq)) * q

    # ------------------------------------------------------------------ #
    # model pieces
    # ------------------------------------------------------------------ #
    def helmholtz(self):
        Ma, Mb, Mc = self.mass()
        Ka, Kb, Kc = self.stiffness()
        a2 = self.alpha ** 2
        return (Ma + a2 * Ka, Mb + a2 * Kb, Mc + a2 * Kc)

    def u_from_m(self, m: np.ndarray) -> np.ndarray:
        """Solve (u, psi) + alpha^2 (u_x, psi_x) = (m, psi) for u (Eq. sde1, first line)."""
        return self.solve(self.helmholtz(), self.apply(self.mass(), m))

    def m_from_u(self, u: np.ndarray) -> np.ndarray:
        """The P1 momentum of a velocity: M m = (M + alpha^2 K) u."""
        return self.solve(self.mass(), self.apply(self.helmholtz(), u))

    def modes(self) -> np.ndarray:
        """xi_k(x_i): [K, n]; k = 2(j-1) is a_j sin(2 pi j x / L), k = 2(j-1)+1 is a_j cos(..)."""
        x = self.x
        out = np.empty((self.K, self.n))
        for jj, a in enumerate(self.amps):
            j = jj + 1
            out[2 * jj] = a * np.sin(2.0 * math.pi * j * x / self.L)
            out[2 * jj + 1] = a * np.cos(2.0 * math.pi * j * x / self.L)
        return out

    def noise(self, dW: np.ndarray, lam=None) -> np.ndarray:
        """Nodal dU of one step from dW, lam: [Q].

        Modes: dU_i = sum_k xi_k(x_i) (dW_k + lambda_k dt).  Matern: w = dW +
        lambda dt on the cells (cell c = [x_c, x_{c+1}]), right-hand side
        eta (dW_h, phi_i) = eta (sqrt(h) / 2) (w_{i-1} + w_i), then k solves with
        M + kappa^{-2} K, the later ones with right-hand side M U_{j-1}.
        """
        w = np.asarray(dW, dtype=np.float64).copy()
        if lam is not None:
            w = w + np.asarray(lam, dtype=np.float64) * self.dt
        if self.noise_model != "matern":
            return self.modes().T @ w
        G = self.matern_operator()
        U = self.solve(G, self.eta * 0.5 * math.sqrt(self.h) * (np.roll(w, 1) + w))
        for _ in range(self.matern_k - 1):
            U = self.solve(G, self.apply(self.mass(), U))
        return U

    def noise_matrix(self) -> np.ndarray:
        """d dU / dw [n, Q] for the increments w = dW + lambda dt of one step: the mode
        functions at the nodes, or the Matern map (G^{-1} M)^{k-1} G^{-1} B, built column
        by column from ``noise`` (it is linear in w)."""
        if self.noise_model != "matern":
            return self.modes().T
        return np.stack([self.noise(e) for e in np.eye(self.n)], axis=1)

    def matern_operator(self):
        """M + kappa^{-2} K, the P1 form of (I - kappa^{-2} d_xx) (Eq. noise_solve2)."""
        Ma, Mb, Mc = self.mass()
        Ka, Kb, Kc = self.stiffness()
        k2 = self.kappa ** -2
        return (Ma + k2 * Ka, Mb + k2 * Kb, Mc + k2 * Kc)

    def residual(self, m1, m0, u1, u0, dU) -> np.ndarray:
        """Assembled residual of Eq. fde1 (second line) for all test functions."""
        mbar = 0.5 * (m0 + m1)
        dv = 0.5 * self.dt * (u0 + u1) + dU
        Ka = self.stiffness()
        return (self.apply(self.mass(), m1 - m0) + self.mu * self.dt * self.apply(Ka, mbar)
                + self.apply(self.advection(dv), mbar))

    def residual_quadrature(self, m1, m0, dU) -> np.ndarray:
        """Eq. fde1 residual by 3-point Gauss quadrature per element (independent check).

        u0, u1 are recomputed from m0, m1 through the Helmholtz relation.
        Integrands are products of two linear functions (or their derivatives),
        so 3-point Gauss is exact and agrees with the closed-form assembly only
        if the assembly is right.
        """
        u0 = self.u_from_m(m0)
        u1 = self.u_from_m(m1)
        h = self.h
        gx = np.array([0.5 - math.sqrt(15) / 10, 0.5, 0.5 + math.sqrt(15) / 10])
        gw = np.array([5.0 / 18, 8.0 / 18, 5.0 / 18])
        mbar = 0.5 * (m0 + m1)
        dm = m1 - m0
        dv = 0.5 * self.dt * (u0 + u1) + dU
        R = np.zeros(self.n)
        for e in range(self.n):
            i0, i1 = e, (e + 1) % self.n
            for xi, wq in zip(gx, gw):
                N = np.array([1.0 - xi, xi])
                dN = np.array([-1.0, 1.0]) / h
                mb = mbar[i0] * N[0] + mbar[i1] * N[1]
                mb_x = mbar[i0] * dN[0] + mbar[i1] * dN[1]
                dmq = dm[i0] * N[0] + dm[i1] * N[1]
                v = dv[i0] * N[0] + dv[i1] * N[1]
                v_x = dv[i0] * dN[0] + dv[i1] * dN[1]
                for r, node in ((0, i0), (1, i1)):
                    integrand = (dmq * N[r] + self.mu * self.dt * mb_x * dN[r]
                                 + mb * v_x * N[r] - mb * v * dN[r])
                    R[node] += wq * h * integrand
        return R

    def step(self, m0: np.ndarray, u0: np.ndarray, dU: np.ndarray):
        """One implicit-midpoint step (Eq. fde1). Returns (m1, u1, iterations, converged)."""
        Ma = self.mass()
        Ka = self.stiffness()
        half_visc = 0.5 * self.mu * self.dt
        m_it = m0.copy()
        u_it = u0.copy()
        if self.scheme == "ea":
            lhs_c = tuple(Ma[j] + half_visc * Ka[j] for j in range(3))
            rhs_c = self.apply(tuple(Ma[j] - half_visc * Ka[j] for j in range(3)), m0)
        for it in range(1, self.max_iter + 1):
            dv = 0.5 * self.dt * (u0 + u_it) + dU
            Aa = self.advection(dv)
            if self.scheme == "ea":
                m_new = self.solve(lhs_c, rhs_c - self.apply(Aa, 0.5 * (m0 + m_it)))
            else:
                lhs = tuple(Ma[j] + half_visc * Ka[j] + 0.5 * Aa[j] for j in range(3))
                rop = tuple(Ma[j] - half_visc * Ka[j] - 0.5 * Aa[j] for j in range(3))
                m_new = self.solve(lhs, self.apply(rop, m0))
            u_new = self.u_from_m(m_new)
            delta = np.max(np.abs(m_new - m_it))
            scale = max(1.0, np.max(np.abs(m_new)))
            m_it, u_it = m_new, u_new
            if delta <= self.tol * scale:
                return m_it, u_it, it, True
        return m_it, u_it, self.max_iter, False

    def window(self, m0: np.ndarray, dW: np.ndarray, lam=None, return_traj: bool = False):
        """Ns steps from m0 with increments dW[s, k] and drift lam[s, k].

        Returns (m_end, u_end, iters[Ns]) and, if ``return_traj``, the list of
        (m, u) after each step (index 0 = start).
        """
        m = np.asarray(m0, dtype=np.float64).copy()
        u = self.u_from_m(m)
        Ns = dW.shape[0]
        iters = np.zeros(Ns, dtype=np.int64)
        conv = True
        traj = [(m.copy(), u.copy())]
        for s in range(Ns):
            dU = self.noise(dW[s], None if lam is None else lam[s])
            m, u, it, ok = self.step(m, u, dU)
            iters[s] = it
            conv = conv and ok
            if return_traj:
                traj.append((m.copy(), u.copy()))
        if return_traj:
            return m, u, iters, conv, traj
        return m, u, iters, conv

    def ensemble_window(self, m0: np.ndarray, dW: np.ndarray, lam=None):
        """Apply ``window`` to every particle: m0 [N, n], dW [N, Ns, Q]."""
        N = m0.shape[0]
        m_out = np.empty_like(m0, dtype=np.float64)
        u_out = np.empty_like(m0, dtype=np.float64)
        iters = np.empty((N, dW.shape[1]), dtype=np.int64)
        conv = np.empty(N, dtype=bool)
        for p in range(N):
            m_out[p], u_out[p], iters[p], conv[p] = self.window(
                m0[p], dW[p], None if lam is None else lam[p])
        return m_out, u_out, iters, conv

    # ------------------------------------------------------------------ #
    # invariants used by the pins
    # ------------------------------------------------------------------ #
    def energy(self, m: np.ndarray) -> float:
        """H = 1/2 (m, u) = 1/2 [(u, u) + alpha^2 (u_x, u_x)] for the P1 pair (m, u)."""
        u = self.u_from_m(m)
        return 0.5 * float(u @ self.apply(self.mass(), m))

    def mass_integral(self, m: np.ndarray) -> float:
        """int m dx = (m, 1)."""
        return float(np.sum(self.apply(self.mass(), m)))

    def exp1_field(self, cells: np.ndarray, a: float, b: float) -> np.ndarray:
        """The initial velocity of Eq. init_solve for one member: U^{0,1} solves
        (U, v) + (U', v') = (|W|, v) for the DG0 field W with cell values ``cells``,
        U^{0,j+1} solves the same with right-hand side (U^{0,j}, v), j = 1, 2, and
        u = a^2 U^{0,3} + b^2."""
        Ma = self.mass()
        Ka = self.stiffness()
        S = tuple(Ma[j] + Ka[j] for j in range(3))
        w = np.abs(np.asarray(cells, dtype=np.float64))
        U = self.solve(S, 0.5 * self.h * (np.roll(w, 1) + w))
        for _ in range(2):
            U = self.solve(S, self.apply(Ma, U))
        return a * a * U + b * b

    def prior_exp1(self, seed: int, N: int, particle0: int = 0):
        """Members particle0 .. particle0 + N - 1 of the initial ensemble of Exp 1 (Sec. 4.1):
        W_p has cell values N(0, h), a_p, b_p ~ N(0, 1), u_p = exp1_field(W_p, a_p, b_p).
        The normals are Philox (seed, TAG_INIT) at counter (k // 4, 0, p, 0): k < n for the
        cells, k = n and n + 1 for a_p and b_p.  Returns the momenta m [N, n] and velocities u [N, n]."""
        from oracle import rng
        p = np.arange(particle0, particle0 + N, dtype=np.uint64)
        z = rng.normals(seed, rng.TAG_INIT, self.n + 2, np.uint64(0), p, np.uint64(0))
        u = np.stack([self.exp1_field(math.sqrt(self.h) * z[q, : self.n], z[q, self.n], z[q, self.n + 1])
                      for q in range(N)])
        m = np.stack([self.m_from_u(uq) for uq in u])
        return m, u

    def prior_sample(self, u_truth: np.ndarray, seed: int, N: int, scale: float):
        """Prior ensemble about a truth velocity (a reading of Eq. init_solve).

        For particle p: W_p is a DG0 field with cell values ~ N(0, h); three
        P1 solves of (I - d_xx) give S^3 W_p; the velocity is
        u_truth + scale (a_p S^3 W_p + b_p) with a_p, b_p ~ N(0, 1).
        Returns the momenta m [N, n] and velocities u [N, n].
        Pinned to its discrete Fourier symbol: the DFT of S^3 W is
        h cos(theta/2) M^2 / G^3 times the half-cell-shifted DFT of the cells, with
        M, G the symbols of the mass matrix and of M + K.
        """
        from oracle import rng
        p = np.arange(N, dtype=np.uint64)
        z = rng.normals(seed, rng.TAG_INIT, self.n + 2, np.uint64(0), p, np.uint64(0))
        Ma = self.mass()
        Ka = self.stiffness()
        smooth = tuple(Ma[j] + Ka[j] for j in range(3))
        u = np.empty((N, self.n))
        for q in range(N):
            cells = math.sqrt(self.h) * z[q, : self.n]          # W on cell e = [x_e, x_{e+1}]
            rhs = 0.5 * self.h * (np.roll(cells, 1) + cells)     # (W, phi_i)
            U = self.solve(smooth, rhs)
            for _ in range(2):
                U = self.solve(smooth, self.apply(Ma, U))
            u[q] = u_truth + scale * (z[q, self.n] * U + z[q, self.n + 1])
        m = np.stack([self.m_from_u(uq) for uq in u])
        return m, u
