"""Host-side analysis of the experiments module (no GPU): the Eq. 7 fit and
the vorticity of a velocity field."""
import numpy as np

from paper_1907_13415_gb300 import experiments as ex


def test_tanh_fit_recovers_eq7_parameters():
    x = np.arange(160.0)
    prof = (0.31 / 2) * (1 - np.tanh((x - 97.25) / (2 * 1.7)))
    xi, sn, lam, rms = ex.tanh_fit(prof, 96.0)
    assert abs(xi - 97.25) < 1e-9 and abs(sn - 0.31) < 1e-9 and abs(lam - 1.7) < 1e-9
    assert rms < 1e-12
    # with S_n and lambda held at other values only x_i moves: to the
    # minimiser of the squared residual over the fit window (|x - 96| < 12),
    # found here by a bounded scalar search on the residual itself
    from scipy.optimize import minimize_scalar
    xi2, sn2, lam2, rms2 = ex.tanh_fit(prof, 96.0, lam=2.0, s_n=1 / 3)
    xs = x[np.abs(x - 96.0) < 12.0]
    ys = prof[np.abs(x - 96.0) < 12.0]

    def cost(c):
        return np.sum(((1 / 6) * (1 - np.tanh((xs - c) / 4.0)) - ys) ** 2)

    best = minimize_scalar(cost, bounds=(94.0, 100.0), method="bounded",
                           options={"xatol": 1e-12})
    assert sn2 == 1 / 3 and lam2 == 2.0 and rms2 > 1e-3
    assert abs(xi2 - best.x) < 1e-6
    # the bias itself: the held curve (S_n = 1/3 > 0.31, lambda = 2 > 1.7)
    # lies above the profile on the nematic side, so the fit moves x_i
    # towards the nematic side, by about 0.4 cells
    assert -0.6 < xi2 - 97.25 < -0.2


def test_vorticity_of_rigid_rotation_and_shear():
    nz, ny, nx = 1, 16, 16
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    k = 2 * np.pi / nx
    u = np.zeros((3, nz, ny, nx))
    u[1, 0] = np.sin(k * x)          # u_y(x): omega = d_x u_y
    om = ex.vorticity(u)[0]
    # central differences of sin: sin(k) cos(k x)
    assert np.allclose(om, np.sin(k) * np.cos(k * x), atol=1e-14)
    u[:] = 0
    u[0, 0] = np.sin(k * y)          # u_x(y): omega = -d_y u_x
    assert np.allclose(ex.vorticity(u)[0], -np.sin(k) * np.cos(k * y), atol=1e-14)
