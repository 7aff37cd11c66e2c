"""Pins of the oracle's t-SURFF flux (Sec. "t-SURFF": the photoelectron amplitude as the time
integral of the Volkov-state current through a surface S).

- A plane wave on the grid: the flux through the box surface is a sum of geometric series
  over each face, written out here in closed form (no loop of the oracle repeated), exact to
  rounding.  It fixes the faces' normals and trapezoid weights, the 1/2 and (2 pi)^(-3/2) of
  the current, the discrete gradient of the orbital and the Volkov factor.
- The Volkov parameters a = -int E, alpha = int a, beta = int |a|^2 of a constant-envelope
  field have closed forms.
- The continuity equation: for a wave packet propagated by the oracle in a field, the flux
  accumulated through an inner surface S minus that through an outer surface S' equals the
  change of the projection on the Volkov state of the shell between them.  The grid version
  holds to the trapezoid rule across the surfaces, O(h^2): checked at two spacings.
"""
import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I


def _axis(n, h):
    return (np.arange(n) - (n - 1) / 2.0) * h


def _trap_series(kappa, x0, h, count):
    """sum_{i<count} tau_i exp(i kappa (x0 + i h)), tau = 1/2 at both ends: geometric series."""
    r = np.exp(1j * kappa * h)
    first, last = np.exp(1j * kappa * x0), np.exp(1j * kappa * (x0 + (count - 1) * h))
    s = first * count if abs(r - 1.0) < 1e-14 else first * (1.0 - r ** count) / (1.0 - r)
    return s - 0.5 * (first + last)


@pytest.mark.parametrize("fd_order", [4, 8])
def test_tsurff_flux_of_a_plane_wave_is_the_closed_form(fd_order):
    n, h, M = 20, 0.35, fd_order // 2
    spec = I.SystemSpec(nx=n, ny=n, nz=n, h=h, fd_order=fd_order, n_orb=1, wells=False, xc=I.XC_NONE,
                        gauge=I.GAUGE_NONE)
    inp = I.make_inputs(spec, with_orbitals=False)
    o = oracle.System(spec, inp)
    x = _axis(n, h)
    q = np.array([0.7, -1.1, 1.6])
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    psi = np.exp(1j * (q[0] * X + q[1] * Y + q[2] * Z)).reshape(1, n, n, n, 1)
    box = (5, 14, 6, 13, 4, 15)
    p = np.array([[0.3, -0.9, 1.2], [1.0, 0.2, -0.4], [-0.6, -1.1, 1.6]])
    a, alpha, beta, t_rel = np.array([0.05, -0.1, 0.2]), np.array([0.3, 0.1, -0.2]), 0.37, 1.3
    got = o.tsurff_flux(psi, box, p, a, alpha, beta, t_rel)[0]
    _, d = oracle.fd_weights(M)
    qd = np.array([2.0 / h * sum(d[m] * np.sin(m * q[ax] * h) for m in range(1, M + 1)) for ax in range(3)])
    want = np.zeros(len(p), dtype=complex)
    for j, pp in enumerate(p):
        k = pp + a
        kappa = q - k
        phase = 0.5 * (pp @ pp * t_rel + 2.0 * pp @ alpha + beta)
        for ax in range(3):
            ua, va = (ax + 1) % 3, (ax + 2) % 3
            tu = _trap_series(kappa[ua], x[box[2 * ua]], h, box[2 * ua + 1] - box[2 * ua] + 1)
            tv = _trap_series(kappa[va], x[box[2 * va]], h, box[2 * va + 1] - box[2 * va] + 1)
            for sgn, c in ((-1.0, box[2 * ax]), (1.0, box[2 * ax + 1])):
                want[j] += (sgn * 0.5 * (2 * np.pi) ** -1.5 * np.exp(1j * phase) * (k[ax] + qd[ax])
                            * np.exp(1j * kappa[ax] * x[c]) * h * h * tu * tv)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_volkov_parameters_of_a_constant_envelope_field():
    E0, w = 0.3, 0.8
    pol = np.array([0.2, -0.4, 0.9])
    spec = I.SystemSpec(nx=8, ny=8, nz=8, h=0.5, n_orb=1, wells=False, xc=I.XC_NONE, gauge=I.GAUGE_LENGTH,
                        amp=E0, omega=w, pol=tuple(pol))
    o = oracle.System(spec, I.make_inputs(spec, with_orbitals=False))
    vol, t, dt = np.zeros(7), 0.0, 0.01
    for _ in range(500):
        vol = o.volkov_step(vol, t, dt)
        t += dt
    c = E0 / w
    a = c * (np.cos(w * t) - 1.0) * pol
    alpha = c * (np.sin(w * t) / w - t) * pol
    beta = c * c * (pol @ pol) * (1.5 * t - 2.0 * np.sin(w * t) / w + np.sin(2.0 * w * t) / (4.0 * w))
    np.testing.assert_allclose(vol[:3], a, rtol=0, atol=1e-10)
    np.testing.assert_allclose(vol[3:6], alpha, rtol=0, atol=1e-10)
    assert vol[6] == pytest.approx(beta, abs=1e-10)


def _outer_weight(n, box):
    """Fraction of each grid point's trapezoid cell outside the box surface."""
    inside = [np.where((np.arange(n) < box[2 * a]) | (np.arange(n) > box[2 * a + 1]), 0.0,
                       np.where((np.arange(n) == box[2 * a]) | (np.arange(n) == box[2 * a + 1]), 0.5, 1.0))
              for a in range(3)]
    return 1.0 - inside[2][:, None, None] * inside[1][None, :, None] * inside[0][None, None, :]


def _shell_identity_error(n, h, S, S2, T=1.0, dt=0.01):
    """max_p |(b_S - b_S') - (P(T) - P(0))| / max_p |P(T) - P(0)| for a Gaussian packet
    (width 0.7, momentum 2 along z) in a length-gauge field, P the shell projection."""
    spec = I.SystemSpec(nx=n, ny=n, nz=n, h=h, fd_order=8, n_orb=1, wells=False, xc=I.XC_NONE,
                        gauge=I.GAUGE_LENGTH, amp=0.3, omega=1.0, pol=(0.3, 0.0, 0.9), dt=dt)
    inp = I.make_inputs(spec, with_orbitals=False)
    x = _axis(n, h)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    w = 0.7
    inp.psi0 = ((np.pi * w * w) ** -0.75 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * w * w))
                * np.exp(2.0j * Z)).reshape(1, n, n, n, 1)
    o = oracle.System(spec, inp)
    ps = np.array([[px, 0.0, pz] for px in (0.0, 0.5) for pz in (1.5, 2.0, 2.5)])
    W = _outer_weight(n, S) - _outer_weight(n, S2)

    def proj(psi, vol, t):
        out = []
        for pp in ps:
            k = pp + vol[:3]
            ph = 0.5 * (pp @ pp * t + 2.0 * pp @ vol[3:6] + vol[6])
            chi = (2 * np.pi) ** -1.5 * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z - ph))
            out.append(np.sum(W * np.conj(chi) * psi[0, ..., 0]) * h ** 3)
        return np.array(out)

    steps = int(round(T / dt))
    psi_t, _, b1, vol, t_rel = o.propagate_tsurff(inp.psi0, 0.0, dt, steps, 1, S, ps, record=False)
    _, _, b2, _, _ = o.propagate_tsurff(inp.psi0, 0.0, dt, steps, 1, S2, ps, record=False)
    dP = proj(psi_t, vol, t_rel) - proj(inp.psi0, np.zeros(7), 0.0)
    return float(np.max(np.abs((b1 - b2)[0] - dP)) / np.max(np.abs(dP)))


def test_tsurff_flux_obeys_the_continuity_equation_to_second_order():
    e1 = _shell_identity_error(40, 0.3, (10, 29) * 3, (4, 35) * 3)
    e2 = _shell_identity_error(55, 0.22, (14, 40) * 3, (6, 48) * 3)
    assert e1 < 2e-2 and e2 < 1e-2, (e1, e2)
    # the residual is the trapezoid rule's across the surfaces: it falls as h^2
    assert 1.5 < e1 / e2 < 2.3, (e1, e2)
