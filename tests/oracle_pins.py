"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` function takes an ``oracle.Oracle`` and returns the worst
deviation it found (0.0 = exact); ``PINS`` maps each name to the function
and the bound it must stay under.  ``test_oracle_pins.py`` runs them on the real oracle,
``test_oracle_mutations.py`` on copies with a planted mistake, each of which
must break at least one pin.

None of the pins re-types the oracle's closed form (Eqs. (cc)/(dd)):
  * the dense pins assemble Saul'yev's equations (aa)/(bb) with the roles of
    the sub-domain decomposition (Sec. 2, k = 1) and solve them;
  * the Fourier pin uses the Cayley form (I - rG)(I + rG)^{-1} of the
    alternating splitting, whose 2x2 blocks are [[1, 2r], [2r, 1]]/(1+2r);
  * the others are invariants (fixed points, mirror symmetry, monotone
    energy) and the exact solution of u_t = u_xx.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

R_VALUES = (0.013, 0.3, 0.5, 1.0, 2.0, 7.25, 1.0e4)


# ---------------------------------------------------------------- references
def saulyev_roles(n: int, parity: int, k: int = 1):
    """Role of every interior node in one step (Sec. 2).

    Paper nodes j = 1..n (node j is array index j-1), walls j = 0 and n+1.
    Odd sub-domains are [x_{2ik}, x_{2ik+k-1}], even ones [x_{2ik+k},
    x_{2(i+1)k-1}]: node j lies in sub-domain floor(j/k), odd when that index
    is even.  First row of each pair of steps (parity 0): odd sub-domains use
    Saul'yev A (new-level neighbour on the left), even ones Saul'yev B
    (new-level neighbour on the right); second row (parity 1): the roles
    swap.  Returns a list of (j, new_nb, old_nb)."""
    roles = []
    for j in range(1, n + 1):
        odd_subdomain = ((j // k) % 2 == 0)
        uses_a = odd_subdomain if parity == 0 else not odd_subdomain
        if uses_a:
            roles.append((j, j - 1, j + 1))   # Eq. (aa)
        else:
            roles.append((j, j + 1, j - 1))   # Eq. (bb)
    return roles


def saulyev_dense_step(u, r, bl, br, parity, exact=False, k=1):
    """One step assembled from Eqs. (aa)/(bb) and solved as a dense system:
    (1+r) u'_j - r u'_{new_nb} = (1-r) u_j + r u_{old_nb}, walls fixed."""
    n = len(u)
    one = Fraction(1) if exact else 1.0
    r = Fraction(r) if exact else float(r)
    cvt = (lambda v: Fraction(v)) if exact else float
    old = {0: cvt(bl), n + 1: cvt(br)}
    for j in range(1, n + 1):
        old[j] = cvt(u[j - 1])
    A = [[0 * one] * n for _ in range(n)]
    rhs = [0 * one] * n
    for (j, new_nb, old_nb) in saulyev_roles(n, parity, k):
        row = j - 1
        A[row][row] = (one + r)
        rhs[row] = (one - r) * old[j] + r * old[old_nb]
        if new_nb == 0 or new_nb == n + 1:
            rhs[row] = rhs[row] + r * old[new_nb]
        else:
            A[row][new_nb - 1] = A[row][new_nb - 1] - r
    if not exact:
        return np.linalg.solve(np.array(A, dtype=np.float64), np.array(rhs))
    # exact Gaussian elimination over the rationals (tiny n only)
    M = [A[i][:] + [rhs[i]] for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def grouping_matrix(n: int, parity: int) -> np.ndarray:
    """G_p: block diagonal of [[1,-1],[-1,1]] on the parity-p groups of the
    decomposition, [1] on its singletons, so that G_0 + G_1 = tridiag(-1,2,-1)
    and a step reads (I + r G_p) u' = (I - r G_{1-p}) u + wall terms."""
    G = np.zeros((n, n))
    roles = {j: nb for (j, nb, _) in saulyev_roles(n, parity)}
    for j in range(1, n + 1):
        nb = roles[j]
        G[j - 1, j - 1] = 1.0
        if 1 <= nb <= n:
            G[j - 1, nb - 1] = -1.0
    return G


def fourier_two_step_eigs(r: float, m_cells: int) -> np.ndarray:
    """Eigenvalues of two periodic steps (parity 0 then 1) on 2*m_cells points.

    In Cayley form each step is C_p = (I - rG_p)(I + rG_p)^{-1}, block
    [[1, 2r], [2r, 1]]/(1+2r) on its groups.  On Bloch waves
    (u_{2m}, u_{2m+1}) = (A, B) e^{i m phi} the parity-0 blocks act as
    S0 = [[1, 2r], [2r, 1]]/(1+2r) and the parity-1 blocks, which couple
    B_m with A_{m+1}, as S1 = [[1, 2r e^{-i phi}], [2r e^{i phi}, 1]]/(1+2r).
    Two steps are similar to C_0 C_1, so their eigenvalues are the roots of
    lam^2 - t lam + rho^2 with t = tr(S0 S1) = (2 + 8 r^2 cos phi)/(1+2r)^2
    and rho = det S0 = (1-2r)/(1+2r), phi = 2 pi k / m_cells."""
    rho = (1.0 - 2.0 * r) / (1.0 + 2.0 * r)
    out = []
    for k in range(m_cells):
        phi = 2.0 * np.pi * k / m_cells
        t = (2.0 + 8.0 * r * r * np.cos(phi)) / (1.0 + 2.0 * r) ** 2
        disc = np.sqrt(complex(t * t - 4.0 * rho * rho))
        out += [(t + disc) / 2.0, (t - disc) / 2.0]
    return np.array(out)


def _rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


# ---------------------------------------------------------------------- pins
def pin_group_vs_2x2_solve(orc) -> float:
    """Eqs. (cc)/(dd) with prefactor 1/(1+2r) solve the group's coupled
    Saul'yev pair: B at the left member, A at the right member (N = 2,
    parity 0 is one group whose outer neighbours are the walls)."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for r in R_VALUES:
        for _ in range(20):
            a, b, c, d = rng.uniform(-1, 1, 4)
            M = np.array([[1 + r, -r], [-r, 1 + r]])
            rhs = np.array([(1 - r) * b + r * a, (1 - r) * c + r * d])
            want = np.linalg.solve(M, rhs)
            got = orc.step(np.array([b, c]), r, a, d, 0)
            worst = max(worst, _rel(got, want) / max(1.0, r))
    return worst


def pin_dense_saulyev(orc) -> float:
    """Whole step == dense solve of Eqs. (aa)/(bb) with the k = 1 roles, for
    every N in 1..17 (odd and even), both parities, several r and walls."""
    rng = np.random.default_rng(12)
    worst = 0.0
    for n in range(1, 18):
        for parity in (0, 1):
            for r in (0.013, 0.5, 1.0, 2.0, 7.25, 300.0):
                u = rng.uniform(-1, 1, n)
                bl, br = rng.uniform(-1, 1, 2)
                want = saulyev_dense_step(u, r, bl, br, parity)
                got = orc.step(u, r, bl, br, parity)
                worst = max(worst, _rel(got, want) / max(1.0, r))
    return worst


def pin_exact_rational(orc) -> float:
    """Tiny cases against exact rational arithmetic (Fractions) of the same
    Saul'yev system: N in 1..6, r in {1/2, 1, 3}, dyadic data."""
    worst = 0.0
    data = [0.5, -1.25, 2.0, 0.75, -0.5, 1.5]
    for n in range(1, 7):
        for parity in (0, 1):
            for r in (0.5, 1.0, 3.0):
                u = np.array(data[:n])
                want = saulyev_dense_step(u, r, 0.25, -0.75, parity, exact=True)
                got = orc.step(u, r, 0.25, -0.75, parity)
                worst = max(worst, _rel(got, np.array([float(v) for v in want])))
    return worst


def pin_run_sequence(orc) -> float:
    """Multi-step runs alternate the groupings from the global step counter:
    run(u, S, step0) == S dense Saul'yev solves of parities step0, step0+1, ..."""
    rng = np.random.default_rng(16)
    worst = 0.0
    for n in (5, 6):
        for step0 in (0, 1, 2, 3):
            for steps in (1, 2, 3, 4):
                u = rng.uniform(-1, 1, n)
                want = u.copy()
                for s in range(steps):
                    want = saulyev_dense_step(want, 1.5, 0.3, -0.4, (step0 + s) % 2)
                got = orc.run(u, 1.5, 0.3, -0.4, steps, step0=step0)
                worst = max(worst, _rel(got, want))
    return worst


def pin_linear_fixed_point(orc) -> float:
    """The linear profile between the wall values is a steady state of the
    heat equation and an exact fixed point of every GE step.  Returns the
    deviation after 7 steps in units of the round-off bound
    7 (2r-1)^2 eps max|u| (each step's rounding is at most (2r-1) eps max|u|,
    the sum of the coefficients' magnitudes, and the step's max-norm is at
    most max(1, 2r-1))."""
    worst = 0.0
    eps = np.finfo(np.float64).eps
    for n in (1, 2, 3, 10, 33, 64):
        for r in R_VALUES:
            bl, br = 0.7, -1.3
            x = np.arange(1, n + 1) / (n + 1.0)
            u = bl + (br - bl) * x
            got = orc.run(u, r, bl, br, 7)
            bound = 7 * max(1.0, 2 * r - 1) ** 2 * eps * np.max(np.abs(u))
            worst = max(worst, float(np.max(np.abs(got - u))) / bound)
    return worst


def pin_mirror_symmetry(orc) -> float:
    """Reflecting the grid swaps the walls.  Even N: the groups of each
    parity map onto themselves; odd N: onto the other parity's groups."""
    rng = np.random.default_rng(13)
    worst = 0.0
    for n in (2, 3, 8, 9, 16, 17):
        for parity in (0, 1):
            for r in (0.3, 2.0, 7.25):
                u = rng.uniform(-1, 1, n)
                bl, br = rng.uniform(-1, 1, 2)
                p_mirror = parity if n % 2 == 0 else 1 - parity
                a = orc.step(u, r, bl, br, parity)[::-1]
                b = orc.step(u[::-1].copy(), r, br, bl, p_mirror)
                worst = max(worst, _rel(a, b) / max(1.0, r))
    return worst


def pin_energy_monotone(orc) -> float:
    """Unconditional stability (Kellogg): with zero walls,
    E_m = ||(I + r G_1) u^{2m}||_2 never increases, for every r > 0.
    Returns the largest relative increase seen (0.0 if monotone)."""
    rng = np.random.default_rng(14)
    worst = 0.0
    for n in (16, 17, 64):
        G1 = grouping_matrix(n, 1)
        for r in (0.05, 0.5, 2.0, 10.0, 1.0e4):
            u = rng.standard_normal(n)
            e_prev = np.linalg.norm(u + r * (G1 @ u))
            for _ in range(40):
                u = orc.run(u, r, 0.0, 0.0, 2)
                e = np.linalg.norm(u + r * (G1 @ u))
                worst = max(worst, (e - e_prev) / e_prev)
                e_prev = e
    return max(worst - 1e-13, 0.0)


def pin_splitting(orc) -> float:
    """Both parities are the alternating splitting of tridiag(-1, 2, -1):
    (I + r G_p) step_p(u) = (I - r G_{1-p}) u for zero walls, with
    G_0 + G_1 = tridiag(-1, 2, -1)."""
    rng = np.random.default_rng(15)
    worst = 0.0
    for n in (1, 2, 5, 8, 13):
        G = [grouping_matrix(n, 0), grouping_matrix(n, 1)]
        T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
        worst = max(worst, float(np.max(np.abs(G[0] + G[1] - T))))
        for parity in (0, 1):
            for r in (0.3, 1.0, 4.0):
                u = rng.uniform(-1, 1, n)
                lhs = (np.eye(n) + r * G[parity]) @ orc.step(u, r, 0.0, 0.0, parity)
                rhs = (np.eye(n) - r * G[1 - parity]) @ u
                worst = max(worst, _rel(lhs, rhs) / max(1.0, r))
    return worst


def pin_fourier_symbol(orc) -> float:
    """Periodic grid: two steps (parity 0 then 1) leave each Bloch space
    {(u_{2m}, u_{2m+1}) = (A, B) e^{i m phi}} invariant.  Their 2x2 symbol T,
    read off by stepping the two basis waves, must have the trace t and the
    determinant rho^2 of ``fourier_two_step_eigs`` (a well-conditioned check:
    no eigenvalue solve of a non-normal matrix).  Deviations are returned in
    units of (2r-1)^2 eps, the round-off scale of two steps."""
    worst = 0.0
    for m_cells in (4, 8, 12):
        n = 2 * m_cells
        m = np.arange(m_cells)
        for r in (0.1, 0.5, 1.0, 3.0, 40.0):
            rho = (1.0 - 2.0 * r) / (1.0 + 2.0 * r)
            for k in range(m_cells):
                phi = 2.0 * np.pi * k / m_cells
                wave = np.exp(1j * m * phi)
                T = np.zeros((2, 2), dtype=complex)
                for col in (0, 1):
                    u = np.zeros(n, dtype=complex)
                    u[col::2] = wave
                    out = orc.run_periodic(u.real, r, 2) + 1j * orc.run_periodic(u.imag, r, 2)
                    T[:, col] = out[0:2]
                t = (2.0 + 8.0 * r * r * np.cos(phi)) / (1.0 + 2.0 * r) ** 2
                unit = max(1.0, 2.0 * r - 1.0) ** 2 * np.finfo(np.float64).eps
                worst = max(worst, abs(np.trace(T) - t) / unit,
                            abs(np.linalg.det(T) - rho * rho) / unit)
                # the rest of each wave is the same symbol times the phase
                for col in (0, 1):
                    u = np.zeros(n, dtype=complex)
                    u[col::2] = wave
                    out = orc.run_periodic(u.real, r, 2) + 1j * orc.run_periodic(u.imag, r, 2)
                    want = np.empty(n, dtype=complex)
                    want[0::2] = T[0, col] * wave
                    want[1::2] = T[1, col] * wave
                    worst = max(worst, float(np.max(np.abs(out - want))) / unit)
    return worst


def pin_exact_solution(orc) -> float:
    """N = 1024, r = 1, 1000 steps from u0 = sin(pi x) with zero walls:
    relative max-norm distance to exp(-pi^2 t) sin(pi x).  The scheme is
    second order at fixed r; this distance is about 8.2e-8."""
    n, r, steps = 1024, 1.0, 1000
    x = np.arange(1, n + 1) / (n + 1.0)
    u = orc.run(np.sin(np.pi * x), r, 0.0, 0.0, steps)
    t = steps * r / (n + 1.0) ** 2
    ex = np.exp(-np.pi ** 2 * t) * np.sin(np.pi * x)
    return _rel(u, ex)


def convergence_ratios(orc, r=1.0, t_final=0.005, intervals=(50, 100, 200, 400)):
    """Error against the exact solution at a fixed final time and fixed r
    for h = 1/M, M in ``intervals`` (odd N = M-1); returns the error ratios
    of successive halvings of h (4 for a second-order scheme)."""
    errs = []
    for M in intervals:
        n = M - 1
        steps = int(round(t_final * M * M / r))
        x = np.arange(1, n + 1) / float(M)
        u = orc.run(np.sin(np.pi * x), r, 0.0, 0.0, steps)
        t = steps * r / float(M * M)
        ex = np.exp(-np.pi ** 2 * t) * np.sin(np.pi * x)
        errs.append(np.max(np.abs(u - ex)) / np.max(np.abs(ex)))
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


def pin_convergence(orc) -> float:
    """Deviation of the halving ratios from [3.5, 4.8] (0.0 inside)."""
    worst = 0.0
    for ratio in convergence_ratios(orc):
        worst = max(worst, max(3.5 - ratio, ratio - 4.8, 0.0))
    return worst


K_VALUES = (2, 3, 4, 5, 16)


def pin_k_dense_saulyev(orc) -> float:
    """General sub-domain width k: the step (confluence pairs by Eqs. (cc)/(dd),
    then Saul'yev A runs left to right and B runs right to left) equals the
    dense solve of Eqs. (aa)/(bb) with the sub-domain roles of Sec. 2."""
    rng = np.random.default_rng(17)
    worst = 0.0
    for k in K_VALUES:
        for n in (1, 2, 3, 7, 15, 16, 17, 33, 40):
            for parity in (0, 1):
                for r in (0.2, 1.0, 6.0):
                    u = rng.uniform(-1, 1, n)
                    bl, br = rng.uniform(-1, 1, 2)
                    want = saulyev_dense_step(u, r, bl, br, parity, k=k)
                    got = orc.step_k(u, r, bl, br, parity, k)
                    worst = max(worst, _rel(got, want) / max(1.0, r))
    return worst


def pin_k1_is_group_step(orc) -> float:
    """Width k = 1 is the 2-point group step, bit for bit (1.0 if not)."""
    rng = np.random.default_rng(18)
    for n in (1, 2, 9, 64):
        for parity in (0, 1):
            u = rng.standard_normal(n)
            if not np.array_equal(orc.step_k(u, 2.5, 0.1, 0.2, parity, 1), orc.step(u, 2.5, 0.1, 0.2, parity)):
                return 1.0
    return 0.0


def pin_k_fixed_point_and_stability(orc) -> float:
    """For every k the linear wall-to-wall profile is a fixed point (in units of
    the round-off bound), and two steps have spectral radius below 1 with
    zero walls (stability for r from 0.5 to 100)."""
    worst = 0.0
    eps = np.finfo(np.float64).eps
    for k in K_VALUES:
        n = 40
        x = np.arange(1, n + 1) / (n + 1.0)
        u = 0.7 + (-1.3 - 0.7) * x
        got = orc.run_k(u, 2.0, 0.7, -1.3, k, 6)
        worst = max(worst, float(np.max(np.abs(got - u))) / (6 * 9 * eps * 1.3))
        for r in (0.5, 4.0, 100.0):
            M = np.zeros((24, 24))
            for j in range(24):
                e = np.zeros(24)
                e[j] = 1.0
                M[:, j] = orc.run_k(e, r, 0.0, 0.0, k, 2)
            rho = float(np.max(np.abs(np.linalg.eigvals(M))))
            worst = max(worst, 0.0 if rho < 1.0 - 1e-6 else 2.0)
    return worst


def pin_k_convergence(orc) -> float:
    """Second order at fixed r for sub-domain widths 4 and 16: halving h
    divides the error by 3.5 to 5 (0.0 inside)."""
    worst = 0.0
    for k in (4, 16):
        errs = []
        for M in (128, 256, 512):
            n = M - 1
            steps = int(round(0.005 * M * M))
            x = np.arange(1, n + 1) / float(M)
            u = orc.run_k(np.sin(np.pi * x), 1.0, 0.0, 0.0, k, steps)
            t = steps / float(M * M)
            ex = np.exp(-np.pi ** 2 * t) * np.sin(np.pi * x)
            errs.append(np.max(np.abs(u - ex)) / np.max(np.abs(ex)))
        for i in range(len(errs) - 1):
            ratio = errs[i] / errs[i + 1]
            worst = max(worst, max(3.5 - ratio, ratio - 5.0, 0.0))
    return worst


PINS = {
    "group_vs_2x2_solve": (pin_group_vs_2x2_solve, 1e-13),
    "dense_saulyev": (pin_dense_saulyev, 1e-12),
    "exact_rational": (pin_exact_rational, 4e-16),
    "run_sequence": (pin_run_sequence, 1e-14),
    "linear_fixed_point": (pin_linear_fixed_point, 1.0),
    "mirror_symmetry": (pin_mirror_symmetry, 1e-14),
    "energy_monotone": (pin_energy_monotone, 0.0),
    "splitting": (pin_splitting, 1e-13),
    "fourier_symbol": (pin_fourier_symbol, 64.0),
    "exact_solution": (pin_exact_solution, 1e-7),
    "convergence": (pin_convergence, 0.0),
    "k_dense_saulyev": (pin_k_dense_saulyev, 1e-12),
    "k1_is_group_step": (pin_k1_is_group_step, 0.0),
    "k_fixed_point_and_stability": (pin_k_fixed_point_and_stability, 1.0),
    "k_convergence": (pin_k_convergence, 0.0),
}
