"""The operator whose residual the mixed-precision grid solves form (five-point Laplacian with
the ghost values of the box condition, minus kappa), checked against the oracle's box solve
(Sec. 4.2, by DST-II / DCT-II): applied to the oracle's solution it gives back the right-hand
side, so the transforms diagonalise exactly that operator. A wrong ghost sign (Dirichlet read
as Neumann or the reverse) fails at the box faces."""
import numpy as np
import pytest

from oracle import kfbi as OK


def five_point(u, h, kappa, neumann):
    """(Delta_h - kappa) u, cell-centred, ghost values u_{-1} = s u_0, u_N = s u_{N-1},
    s = +1 (Neumann, DCT-II) or -1 (Dirichlet, DST-II)."""
    s = 1.0 if neumann else -1.0
    g = np.pad(u, 1)
    g[0, 1:-1] = s * u[0]
    g[-1, 1:-1] = s * u[-1]
    g[1:-1, 0] = s * u[:, 0]
    g[1:-1, -1] = s * u[:, -1]
    lap = (g[1:-1, :-2] + g[1:-1, 2:] + g[:-2, 1:-1] + g[2:, 1:-1] - 4.0 * u) / (h * h)
    return lap - kappa * u


@pytest.mark.parametrize("N", [8, 32, 64])
@pytest.mark.parametrize("boxbc,kappa", [(OK.BOX_DIRICHLET0, 0.0), (OK.BOX_DIRICHLET0, 40.0),
                                         (OK.BOX_NEUMANN0, 20.0), (OK.BOX_NEUMANN0, 3000.0)])
def test_box_solve_inverts_the_five_point_operator(N, boxbc, kappa):
    rng = np.random.default_rng(N + boxbc)
    g = OK.Grid(N, (-1.0, 1.0, -1.0, 1.0))
    C = rng.standard_normal((N, N))
    u = OK.solve_grid(g, C, kappa, boxbc)
    back = five_point(u, g.h, kappa, boxbc == OK.BOX_NEUMANN0)
    assert np.abs(back - C).max() < 1e-9 * np.abs(C).max()
    # the other ghost sign does not reproduce C at the faces
    wrong = five_point(u, g.h, kappa, boxbc != OK.BOX_NEUMANN0)
    assert np.abs(wrong - C).max() > 1e-3 * np.abs(C).max()


def test_one_refinement_step_in_float32_arithmetic():
    """The refinement the GPU path runs, written with numpy: a float32 box solve (the oracle's
    solve with its input and output rounded to float32), then r = C - (Delta_h - kappa) u in
    float64 and u += the float32 solve of r: the error drops from float32 level to well below
    it (a plausible sign error in the residual would make it grow)."""
    N, kappa = 64, 300.0
    g = OK.Grid(N, (-1.0, 1.0, -1.0, 1.0))
    C = np.random.default_rng(5).standard_normal((N, N))
    exact = OK.solve_grid(g, C, kappa, OK.BOX_NEUMANN0)

    def solve32(f):
        return OK.solve_grid(g, f.astype(np.float32).astype(np.float64), kappa, OK.BOX_NEUMANN0).astype(np.float32)

    u = solve32(C).astype(np.float64)
    e0 = np.abs(u - exact).max() / np.abs(exact).max()
    r = C - five_point(u, g.h, kappa, True)
    u = u + solve32(r).astype(np.float64)
    e1 = np.abs(u - exact).max() / np.abs(exact).max()
    assert 1e-9 < e0 < 1e-5
    assert e1 < 1e-3 * e0
