"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test checks the oracle against something other than itself: exact rational FD
weights, an independent weight recursion, the discrete plane-wave spectrum, polynomial
exactness and the known truncation term, the exact norm and energy identities of the
truncated Taylor series, free-Gaussian spreading, harmonic-oscillator (Ehrenfest)
dynamics, a dense brute-force projector matrix, the Dirac exchange coefficient and the
functional derivative of E_x.
"""
import dataclasses
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spec(**kw):
    base = dict(nx=10, ny=12, nz=14, h=0.4, fd_order=4, bc=I.BC_ZERO, n_orb=2, n_atoms=0,
                projectors=False, wells=False, xc=I.XC_NONE, gauge=I.GAUGE_NONE, amp=0.0)
    base.update(kw)
    return I.SystemSpec(**base)


def _inputs(spec, vloc=None):
    inp = I.make_inputs(spec, with_orbitals=False)
    if vloc is not None:
        inp.vloc = vloc
    return inp


def _axis(spec, n):
    return I._axis(n, spec.h, spec.bc)


def _grids(spec):
    x, y, z = _axis(spec, spec.nx), _axis(spec, spec.ny), _axis(spec, spec.nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _inner(a, b, h):
    return np.vdot(a, b) * h ** 3


# ---------------------------------------------------------------------------------
# Finite-difference weights
# ---------------------------------------------------------------------------------

def _read_golden():
    rows = {}
    with open(os.path.join(GOLDEN, "fd_weights.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            kind, order, *w = line.split()
            rows[(kind, int(order))] = [Fraction(v) for v in w]
    return rows


def _fornberg(z, x, m):
    """Weights c[j][k] of the k-th derivative at z from nodes x (Fornberg's recursion,
    SIAM Review 40 (1998) 685), in exact rational arithmetic."""
    n = len(x) - 1
    c = [[Fraction(0)] * (m + 1) for _ in range(n + 1)]
    c1, c4 = Fraction(1), x[0] - z
    c[0][0] = Fraction(1)
    for i in range(1, n + 1):
        mn = min(i, m)
        c2, c5, c4 = Fraction(1), c4, x[i] - z
        for j in range(i):
            c3 = x[i] - x[j]
            c2 = c2 * c3
            if j == i - 1:
                for k in range(mn, 0, -1):
                    c[i][k] = c1 * (k * c[i - 1][k - 1] - c5 * c[i - 1][k]) / c2
                c[i][0] = -c1 * c5 * c[i - 1][0] / c2
            for k in range(mn, 0, -1):
                c[j][k] = (c4 * c[j][k] - k * c[j][k - 1]) / c3
            c[j][0] = c4 * c[j][0] / c3
        c1 = c2
    return c


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_fd_weights_match_golden_and_fornberg(M):
    gold = _read_golden()
    c, d = oracle.fd_weights(M)
    lap, grad = gold[("lap", 2 * M)], gold[("grad", 2 * M)]
    np.testing.assert_allclose(c, [float(v) for v in lap], rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(d, [float(v) for v in grad], rtol=1e-15, atol=1e-16)
    nodes = [Fraction(m) for m in range(-M, M + 1)]
    w = _fornberg(Fraction(0), nodes, 2)
    for m in range(0, M + 1):
        assert w[M + m][2] == lap[m]
        if m > 0:
            assert w[M + m][1] == grad[m] and w[M - m][1] == -grad[m]


# ---------------------------------------------------------------------------------
# Kinetic operator: plane waves (Bloch), polynomials (finite box)
# ---------------------------------------------------------------------------------

def _plane_wave_case(fd_order, gauge, seed=5):
    spec = _spec(bc=I.BC_BLOCH, fd_order=fd_order, n_orb=3, n_k=2, gauge=gauge, amp=0.3,
                 omega=0.7, pol=(0.3, -0.5, 0.8), seed=seed)
    inp = _inputs(spec)
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    X, Y, Z = _grids(spec)
    G = np.array([[0, 0, 0], [1, -2, 3], [-3, 4, 5]])
    psi = np.empty((2, spec.nz, spec.ny, spec.nx, 3), dtype=np.complex128)
    qs = np.empty((2, 3, 3))
    for ik in range(2):
        for o in range(3):
            q = inp.kpts[ik] + 2 * np.pi * G[o] / L
            qs[ik, o] = q
            psi[ik, ..., o] = np.exp(1j * (q[0] * X + q[1] * Y + q[2] * Z))
    return spec, inp, psi, qs


def _pw_eigen(spec, q, A):
    M = spec.fd_order // 2
    c, d = oracle.fd_weights(M)
    h = spec.h
    kin = sum((-c[0] - 2 * sum(c[m] * math.cos(m * qa * h) for m in range(1, M + 1))) / (2 * h * h)
              for qa in q)
    grad = np.array([2.0 / h * sum(d[m] * math.sin(m * qa * h) for m in range(1, M + 1)) for qa in q])
    return kin + float(np.dot(A, grad)) + 0.5 * float(np.dot(A, A)), grad


@pytest.mark.parametrize("fd_order", [4, 8])
@pytest.mark.parametrize("gauge", [I.GAUGE_NONE, I.GAUGE_VELOCITY])
def test_plane_wave_spectrum(fd_order, gauge):
    spec, inp, psi, qs = _plane_wave_case(fd_order, gauge)
    o = oracle.System(spec, inp)
    t = math.pi / (2 * spec.omega)  # sin(omega t) = 1 -> A = amp * pol
    E, A = o.field(t)
    if gauge == I.GAUGE_VELOCITY:
        np.testing.assert_allclose(A, spec.amp * np.array(spec.pol), rtol=1e-14)
    hpsi = o.apply_H(psi, t=t)
    for ik in range(2):
        for j in range(3):
            lam, _ = _pw_eigen(spec, qs[ik, j], A)
            np.testing.assert_allclose(hpsi[ik, ..., j], lam * psi[ik, ..., j], rtol=0, atol=1e-11 * max(1, abs(lam)))


@pytest.mark.parametrize("fd_order", [4, 8])
def test_polynomial_exactness_and_truncation_term(fd_order):
    M = fd_order // 2
    spec = _spec(nx=2 * M + 3, ny=2 * M + 5, nz=2 * M + 3, h=0.37, fd_order=fd_order, n_orb=1)
    o = oracle.System(spec, _inputs(spec))
    X, Y, Z = _grids(spec)
    p = 2 * M + 1
    # degree <= 2M+1: exact.  f = x^p + 0.3 x^2 y^(p-2) + y^3 z^2 - 1.7 z^p
    f = X ** p + 0.3 * X ** 2 * Y ** (p - 2) + Y ** 3 * Z ** 2 - 1.7 * Z ** p
    lap = (p * (p - 1) * X ** (p - 2) + 0.6 * Y ** (p - 2) + 0.3 * (p - 2) * (p - 3) * X ** 2 * Y ** (p - 4)
           + 6 * Y * Z ** 2 + 2 * Y ** 3 - 1.7 * p * (p - 1) * Z ** (p - 2))
    out = o.apply_H(f[None, ..., None])[0, ..., 0]
    sl = (slice(M, spec.nz - M), slice(M, spec.ny - M), slice(M, spec.nx - M))
    np.testing.assert_allclose(out[sl], -0.5 * lap[sl], rtol=1e-9, atol=1e-9 * np.abs(lap).max())
    # degree 2M+2 at the box centre (x = 0): Lap_h x^(2M+2) = 2 h^(2M) sum_m c_m m^(2M+2) != 0
    q = 2 * M + 2
    g = X ** q
    c, _ = oracle.fd_weights(M)
    expect = 2 * spec.h ** (q - 2) * sum(c[m] * m ** q for m in range(1, M + 1))
    cz, cy, cx = spec.nz // 2, spec.ny // 2, spec.nx // 2
    assert abs(X[cz, cy, cx]) < 1e-15
    got = o.apply_H(g[None, ..., None])[0, cz, cy, cx, 0]
    assert abs(expect) > 1e-6
    np.testing.assert_allclose(got.real, -0.5 * expect, rtol=1e-10)


# ---------------------------------------------------------------------------------
# Hermiticity of every term
# ---------------------------------------------------------------------------------

def _full_case(bc, seed=11):
    if bc == I.BC_ZERO:
        spec = _spec(nx=14, ny=13, nz=12, h=0.35, fd_order=8, n_orb=3, n_atoms=3, projectors=True,
                     wells=True, xc=I.XC_LDA_X, gauge=I.GAUGE_LENGTH, amp=0.05, omega=0.3,
                     envelope=I.ENV_SIN2, t_total=10.0, seed=seed)
    else:
        spec = _spec(nx=12, ny=12, nz=12, h=0.4, fd_order=4, bc=I.BC_BLOCH, n_orb=2, n_k=3,
                     n_atoms=2, projectors=True, wells=True, xc=I.XC_LDA_X,
                     gauge=I.GAUGE_VELOCITY, amp=0.2, omega=0.3, pol=(0.2, 0.3, 0.9),
                     lattice="random", seed=seed)
    inp = I.make_inputs(spec)
    if bc == I.BC_BLOCH:
        inp.pos = inp.pos + np.array([0.4, 2.3, 4.4])  # atoms near the cell faces: wrapped spheres
    return spec, inp


@pytest.mark.parametrize("bc", [I.BC_ZERO, I.BC_BLOCH])
def test_hermiticity(bc):
    spec, inp = _full_case(bc)
    o = oracle.System(spec, inp)
    phi = I.random_orbitals(spec, 1)
    psi = I.random_orbitals(spec, 2)
    vx = o.vx_of(inp.psi0)
    t = 1.3
    hphi = o.apply_H(phi, t, vx)
    hpsi = o.apply_H(psi, t, vx)
    for ik in range(phi.shape[0]):
        for j in range(spec.n_orb):
            a = _inner(phi[ik, ..., j], hpsi[ik, ..., j], spec.h)
            b = np.conj(_inner(psi[ik, ..., j], hphi[ik, ..., j], spec.h))
            assert abs(a - b) <= 1e-12 * abs(a)


# ---------------------------------------------------------------------------------
# Projectors: dense brute force and closed-form Gaussian integrals
# ---------------------------------------------------------------------------------

def _dense_vnl(spec, inp, k, A):
    """Brute-force N x N matrix sum_aj |b_aj> D_aj <b_aj| h^3 built point by point over
    every image of every atom in a 3x3x3 block of cells."""
    N = spec.n_points
    V = np.zeros((N, N), dtype=np.complex128)
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    x, y, z = (_axis(spec, n) for n in (spec.nx, spec.ny, spec.nz))
    shifts = [np.zeros(3)] if spec.bc == I.BC_ZERO else [
        np.array([a, b, c]) * L for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    for a in range(inp.pos.shape[0]):
        # one Bloch projector per (a, j): the images of the sphere add into one vector
        vec = [np.zeros(N, dtype=np.complex128) for _ in range(4)]
        for T in shifts:
            for iz in range(spec.nz):
                for iy in range(spec.ny):
                    for ix in range(spec.nx):
                        u = np.array([x[ix], y[iy], z[iz]]) + T  # point image at r + T
                        dvec = u - inp.pos[a]
                        r2 = float(dvec @ dvec)
                        if r2 > spec.r_cut ** 2:
                            continue
                        g = math.exp(-r2 / (2 * spec.r_c ** 2))
                        # psi(u) = exp(i k.T) psi(r); gauge factor exp(i A.d)
                        ph = np.exp(1j * (k @ T + A @ dvec))
                        p = (iz * spec.ny + iy) * spec.nx + ix
                        for j, b in enumerate((g, dvec[0] * g, dvec[1] * g, dvec[2] * g)):
                            vec[j][p] += b * ph
        for j in range(4):
            V += inp.D[a, j] * spec.h ** 3 * np.outer(np.conj(vec[j]), vec[j])
    return V


@pytest.mark.parametrize("bc", [I.BC_ZERO, I.BC_BLOCH])
def test_projectors_dense_bruteforce(bc):
    if bc == I.BC_ZERO:
        spec = _spec(nx=8, ny=8, nz=8, h=0.45, n_orb=2, n_atoms=2, projectors=True, seed=3)
    else:
        spec = _spec(nx=8, ny=8, nz=8, h=0.45, bc=I.BC_BLOCH, n_orb=2, n_k=2, n_atoms=2,
                     projectors=True, gauge=I.GAUGE_VELOCITY, amp=0.4, omega=0.5,
                     pol=(0.6, 0.0, 0.8), seed=3)
    inp = I.make_inputs(spec)
    if bc == I.BC_BLOCH:
        inp.pos = np.array([[0.1, 0.2, 3.4], [3.3, 1.7, 0.05]])  # spheres cross cell faces
    t = 0.9
    o_with = oracle.System(spec, inp)
    o_without = oracle.System(spec, inp, projectors=False)
    _, A = o_with.field(t)
    psi = I.random_orbitals(spec, 9)
    vnl = o_with.apply_H(psi, t) - o_without.apply_H(psi, t)
    for ik in range(psi.shape[0]):
        V = _dense_vnl(spec, inp, inp.kpts[ik], A)
        assert np.allclose(V, V.conj().T, atol=1e-14)
        assert np.linalg.matrix_rank(V, tol=1e-10) <= 4 * inp.pos.shape[0]
        for j in range(spec.n_orb):
            ref = V @ psi[ik, ..., j].reshape(-1)
            np.testing.assert_allclose(vnl[ik, ..., j].reshape(-1), ref, rtol=0,
                                       atol=1e-12 * np.abs(ref).max())


def test_projector_gaussian_integrals():
    """<b_1|b_1> = int_(r<=R) g^2 and <b_2|b_2> = int_(r<=R) x^2 g^2, radial integrals
    over the cut sphere (the full-space values are pi^(3/2) r_c^3 and pi^(3/2) r_c^5/2);
    the grid sum at h = 0.1 matches them to better than 1e-4."""
    from scipy.integrate import quad
    spec = _spec(nx=41, ny=41, nz=41, h=0.1, n_orb=1, n_atoms=1, projectors=True)
    inp = I.make_inputs(spec, with_orbitals=False)
    inp.pos = np.zeros((1, 3))
    X, Y, Z = _grids(spec)
    g = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * spec.r_c ** 2))
    g[(X ** 2 + Y ** 2 + Z ** 2) > spec.r_cut ** 2] = 0.0
    a2, R = spec.r_c ** 2, spec.r_cut
    i0 = quad(lambda r: 4 * math.pi * r * r * math.exp(-r * r / a2), 0, R, epsabs=0, epsrel=1e-13)[0]
    i2 = quad(lambda r: 4 * math.pi / 3 * r ** 4 * math.exp(-r * r / a2), 0, R, epsabs=0, epsrel=1e-13)[0]
    assert abs(i0 / (math.pi ** 1.5 * spec.r_c ** 3) - 1) < 1e-4
    assert abs(i2 / (math.pi ** 1.5 * spec.r_c ** 5 / 2) - 1) < 1e-3
    for j, (b, exact) in enumerate([(g, i0), (X * g, i2)]):
        inp.D = np.zeros((1, 4))
        inp.D[0, j] = 1.0
        o1 = oracle.System(spec, inp)
        o0 = oracle.System(spec, inp, projectors=False)
        psi = b[None, ..., None].astype(np.complex128)
        out = (o1.apply_H(psi) - o0.apply_H(psi))[0, ..., 0]
        # V_NL b = b <b|b>
        ratio = np.vdot(b, out).real / np.vdot(b, b).real
        assert abs(ratio / exact - 1) < 1e-4, (ratio, exact)
    assert o1.sphere_count(0) == int(((X ** 2 + Y ** 2 + Z ** 2) <= spec.r_cut ** 2).sum())


# ---------------------------------------------------------------------------------
# Taylor step: eigenvector, exact norm and energy identities
# ---------------------------------------------------------------------------------

def test_taylor_on_eigenvector():
    spec, inp, psi, qs = _plane_wave_case(8, I.GAUGE_NONE)
    o = oracle.System(spec, inp)
    dt = 0.03
    out = o.taylor_substep(psi, 0.0, dt)
    for ik in range(2):
        for j in range(3):
            lam, _ = _pw_eigen(spec, qs[ik, j], np.zeros(3))
            z = -1j * dt * lam
            R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
            np.testing.assert_allclose(out[ik, ..., j], R * psi[ik, ..., j], rtol=0, atol=1e-12)


@pytest.mark.parametrize("bc", [I.BC_ZERO, I.BC_BLOCH])
def test_norm_and_energy_identities(bc):
    """For Hermitian H frozen over the step, |R(-i tau x)|^2 = 1 - x^6/72 + x^8/576, so
    ||psi'||^2 = ||psi||^2 - tau^6/72 ||H^3 psi||^2 + tau^8/576 ||H^4 psi||^2 and
    <psi'|H|psi'> = <H> - tau^6/72 <H^3psi|H|H^3psi> + tau^8/576 <H^4psi|H|H^4psi>."""
    spec, inp = _full_case(bc)
    o = oracle.System(spec, inp)
    psi = I.random_orbitals(spec, 4) * 0.05
    t, tau = 0.7, 0.02
    vx = o.vx_of(psi)
    out = o.taylor_substep(psi, t, tau)
    H = lambda v: o.apply_H(v, t + tau / 2, vx)
    h1 = H(psi)
    h2 = H(h1)
    h3 = H(h2)
    h4 = H(h3)
    h3h, h4h = H(h3), H(h4)
    hout = H(out)
    for ik in range(psi.shape[0]):
        for j in range(spec.n_orb):
            s = (ik, Ellipsis, j)
            n0 = _inner(psi[s], psi[s], spec.h).real
            n1 = _inner(out[s], out[s], spec.h).real
            c6 = _inner(h3[s], h3[s], spec.h).real
            c8 = _inner(h4[s], h4[s], spec.h).real
            pred = n0 - tau ** 6 / 72 * c6 + tau ** 8 / 576 * c8
            assert abs(n1 - n0) > 1e-6 * n0  # the high-order terms are visible
            assert abs(n1 - pred) <= 1e-12 * n0
            e0 = _inner(psi[s], h1[s], spec.h).real
            e1 = _inner(out[s], hout[s], spec.h).real
            epred = (e0 - tau ** 6 / 72 * _inner(h3[s], h3h[s], spec.h).real
                     + tau ** 8 / 576 * _inner(h4[s], h4h[s], spec.h).real)
            assert abs(e1 - epred) <= 1e-11 * abs(e0)


# ---------------------------------------------------------------------------------
# Dynamics with closed forms: free Gaussian, harmonic oscillator (Ehrenfest)
# ---------------------------------------------------------------------------------

def test_free_gaussian_spreading():
    a = 1.0
    spec = _spec(nx=47, ny=47, nz=47, h=0.25, fd_order=8, n_orb=1)
    o = oracle.System(spec, _inputs(spec))
    X, Y, Z = _grids(spec)
    psi = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * a * a)).astype(np.complex128)
    psi /= math.sqrt(np.vdot(psi, psi).real * spec.h ** 3)
    psi = psi[None, ..., None]
    dt, nst = 0.01, 100
    out, _ = o.propagate(psi, 0.0, dt, nst, 1, record=False)
    n = o.density(out)
    t = dt * nst
    expect = a * a / 2 * (1 + t * t / a ** 4)
    for C in (X, Y, Z):
        got = (C ** 2 * n).sum() / n.sum()
        assert abs(got / expect - 1) < 2e-6, (got, expect)


def _ho_case(E0=0.0, omega=0.0):
    w0, z0 = 1.0, 0.5
    spec = _spec(nx=41, ny=41, nz=49, h=0.25, fd_order=8, n_orb=1,
                 gauge=I.GAUGE_LENGTH if E0 else I.GAUGE_NONE, amp=E0, omega=omega)
    X, Y, Z = _grids(spec)
    v = 0.5 * w0 ** 2 * (X ** 2 + Y ** 2 + Z ** 2)
    o = oracle.System(spec, _inputs(spec, vloc=v))
    psi = np.exp(-w0 * (X ** 2 + Y ** 2 + (Z - z0) ** 2) / 2).astype(np.complex128)
    psi /= math.sqrt(np.vdot(psi, psi).real * spec.h ** 3)
    return spec, o, psi[None, ..., None], w0, z0


def test_harmonic_oscillator_coherent_state():
    spec, o, psi, w0, z0 = _ho_case()
    dt, nst = 0.01, 150
    _, obs = o.propagate(psi, 0.0, dt, nst, 1)
    t = obs[:, 0]
    zt = obs[:, 6] / (spec.occ * obs[:, 1])
    np.testing.assert_allclose(zt, z0 * np.cos(w0 * t), atol=2e-6)
    np.testing.assert_allclose(obs[:, 4:6], 0.0, atol=1e-12)
    np.testing.assert_allclose(obs[:, 1], 1.0, atol=1e-9)


def test_harmonic_oscillator_driven_ehrenfest():
    """Quadratic V: <z> obeys z'' = -w0^2 z - E(t) exactly (charge -1, +E.r coupling)."""
    E0, om = 0.05, 0.6
    spec, o, psi, w0, z0 = _ho_case(E0, om)
    dt, nst = 0.01, 150
    _, obs = o.propagate(psi, 0.0, dt, nst, 1)
    t = obs[:, 0]
    zt = obs[:, 6] / (spec.occ * obs[:, 1])
    exact = z0 * np.cos(w0 * t) + E0 / (w0 ** 2 - om ** 2) * (om / w0 * np.sin(w0 * t) - np.sin(om * t))
    np.testing.assert_allclose(zt, exact, atol=3e-6)
    # the field record is E_z at the first sub-step midpoint
    np.testing.assert_allclose(obs[:, 7], E0 * np.sin(om * (t + dt / 2)), rtol=1e-13, atol=1e-16)
    # two sub-steps of dt/2 per configured step: same trajectory, field at t + dt/4
    _, obs2 = o.propagate(psi, 0.0, 2 * dt, nst // 2, 2)
    t2 = obs2[:, 0]
    np.testing.assert_allclose(t2, t[::2], rtol=1e-14)
    z2 = obs2[:, 6] / (spec.occ * obs2[:, 1])
    exact2 = z0 * np.cos(w0 * t2) + E0 / (w0 ** 2 - om ** 2) * (om / w0 * np.sin(w0 * t2) - np.sin(om * t2))
    np.testing.assert_allclose(z2, exact2, atol=3e-6)
    np.testing.assert_allclose(obs2[:, 7], E0 * np.sin(om * (t2 + dt / 2)), rtol=1e-13, atol=1e-16)


def test_sin2_envelope_length_gauge():
    T = 40.0
    spec = _spec(gauge=I.GAUGE_LENGTH, amp=0.005, omega=0.057, envelope=I.ENV_SIN2, t_total=T)
    o = oracle.System(spec, _inputs(spec))
    for t, env in ((0.0, 0.0), (T / 2, 1.0), (T / 4, 0.5), (T, 0.0), (T + 1, 0.0)):
        E, A = o.field(t)
        np.testing.assert_allclose(E, [0, 0, spec.amp * env * math.sin(spec.omega * t)], atol=1e-18)
        assert np.all(A == 0)


# ---------------------------------------------------------------------------------
# Field, LDA exchange, density, dipole, energy bookkeeping
# ---------------------------------------------------------------------------------

def test_velocity_gauge_field_is_minus_dA_dt():
    spec = _spec(gauge=I.GAUGE_VELOCITY, amp=0.2, omega=0.03, envelope=I.ENV_SIN2, t_total=80.0,
                 pol=(0.0, 0.6, 0.8))
    o = oracle.System(spec, _inputs(spec))
    for t in (3.0, 17.5, 41.0, 79.0):
        eps = 1e-5
        _, Ap = o.field(t + eps)
        _, Am = o.field(t - eps)
        E, _ = o.field(t)
        np.testing.assert_allclose(E, -(Ap - Am) / (2 * eps), rtol=1e-8, atol=1e-13)
    E, A = o.field(100.0)
    assert np.all(A == 0) and np.all(E == 0)


def test_lda_exchange_dirac_coefficient_and_derivative():
    spec = _spec(nx=6, ny=5, nz=4, xc=I.XC_LDA_X)
    o = oracle.System(spec, _inputs(spec))
    n0 = 0.37
    n = np.full(spec.n_points, n0)
    ex, vx = o.lda_x(n)
    C_x = 0.7385587663820224  # Dirac exchange constant (3/4)(3/pi)^(1/3)
    vol = spec.n_points * spec.h ** 3
    np.testing.assert_allclose(ex, -C_x * n0 ** (4 / 3) * vol, rtol=1e-14)
    rng = np.random.default_rng(3)
    n = rng.uniform(0.01, 1.0, spec.n_points)
    _, vx = o.lda_x(n)
    for p in (0, 7, 33, 100):
        d = 1e-5
        npl, nmi = n.copy(), n.copy()
        npl[p] += d
        nmi[p] -= d
        der = (o.lda_x(npl)[0] - o.lda_x(nmi)[0]) / (2 * d * spec.h ** 3)
        np.testing.assert_allclose(der, vx[p], rtol=1e-8)


def test_density_and_dipole_of_shifted_gaussian():
    spec = _spec(nx=41, ny=41, nz=41, h=0.3, n_orb=1, xc=I.XC_NONE)
    o = oracle.System(spec, _inputs(spec))
    X, Y, Z = _grids(spec)
    c = np.array([0.7, -1.1, 0.4])
    psi = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / 2).astype(np.complex128)
    psi /= math.sqrt(np.vdot(psi, psi).real * spec.h ** 3)
    obs = o.observables(psi[None, ..., None], 0.0, 0.0)
    np.testing.assert_allclose(obs[1], 1.0, rtol=1e-13)
    np.testing.assert_allclose(obs[4:7], spec.occ * c, rtol=1e-9)
    n = o.density(psi[None, ..., None])
    np.testing.assert_allclose(n.sum() * spec.h ** 3, spec.occ, rtol=1e-13)


def test_energy_and_current_of_plane_waves_with_exchange():
    """Plane waves have uniform density n0, so every term is closed form:
    E = sum f (lam + v_x(n0)) - n0 v_x(n0) V + E_x,   J = -(1/V) sum f (g(q) + A)."""
    spec, inp, psi, qs = _plane_wave_case(4, I.GAUGE_VELOCITY)
    spec = dataclasses.replace(spec, xc=I.XC_LDA_X)
    o = oracle.System(spec, inp)
    vol = spec.n_points * spec.h ** 3
    psi = psi / math.sqrt(vol)
    t = 0.4
    obs = o.observables(psi, 0.0, t)
    _, A = o.field(t)
    n0 = spec.occ * spec.n_orb * inp.kw.sum() / vol
    vx0 = -(3 * n0 / math.pi) ** (1 / 3)
    ex = -0.75 * (3 * n0 / math.pi) ** (1 / 3) * n0 * vol
    eb, J = 0.0, np.zeros(3)
    for ik in range(2):
        for j in range(3):
            lam, g = _pw_eigen(spec, qs[ik, j], A)
            eb += inp.kw[ik] * spec.occ * (lam + vx0)
            J += inp.kw[ik] * spec.occ * (g + A)
    np.testing.assert_allclose(obs[3], ex, rtol=1e-13)
    np.testing.assert_allclose(obs[2], eb - n0 * vx0 * vol + ex, rtol=1e-12)
    np.testing.assert_allclose(obs[4:7], -J / vol, rtol=1e-12, atol=1e-15)


def test_energy_conservation_at_zero_field():
    """Zero field.  Without the exchange term H is fixed and the Taylor-4 energy error per
    step is O(dt^6) (norm/energy identities), so over a fixed time the drift falls >= 16x
    when dt halves.  With the exchange term frozen over each step the scheme is
    first order in the density, so the drift falls ~2x when dt halves."""
    spec = _spec(nx=16, ny=16, nz=16, h=0.35, fd_order=4, n_orb=2, n_atoms=2, wells=True,
                 xc=I.XC_LDA_X, seed=6)
    inp = I.make_inputs(spec)
    for xc, factor in ((I.XC_NONE, 16.0), (I.XC_LDA_X, 1.8)):
        o = oracle.System(spec, inp, xc=xc)
        drifts = []
        for dt, nst in ((0.02, 20), (0.01, 40)):
            _, obs = o.propagate(inp.psi0, 0.0, dt, nst, 1)
            psi_end, _ = o.propagate(inp.psi0, 0.0, dt, nst, 1, record=False)
            e_end = o.observables(psi_end, dt * nst, dt * nst)[2]
            drifts.append(abs(e_end - obs[0, 2]))
        assert drifts[0] < 2e-3 * abs(obs[0, 2])
        assert drifts[1] * factor < drifts[0], (xc, drifts)


# ---------------------------------------------------------------------------------------
# CFM4 (Sec. "New propagators for real-time TDDFT": two exponentials with the Hamiltonian
# at the Gauss points t1,2 = t + (1/2 -+ sqrt3/6) dt, weights a1,2 = (3 -+ 2 sqrt3)/12)
# ---------------------------------------------------------------------------------------
def _golden_cfm4():
    """The paper's printed CFM4 constants (tests/golden/cfm4_constants.txt)."""
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "cfm4_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                name, expr = (x.strip() for x in line.split("=", 1))
                out[name] = eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt})
    return out


def test_cfm4_constants_and_exchange_extrapolation():
    """The constants are the printed ones; the history weights are Lagrange extrapolation
    (exact on polynomials of degree nh - 1, summing to one), combined with the a's."""
    (a1, a2), (th1, th2) = oracle.cfm4_constants()
    g = _golden_cfm4()
    assert a1 == pytest.approx(g["alpha1"], abs=1e-16) and a2 == pytest.approx(g["alpha2"], abs=1e-16)
    assert th1 == pytest.approx(g["theta1"], abs=1e-16) and th2 == pytest.approx(g["theta2"], abs=1e-16)
    assert a1 + a2 == pytest.approx(0.5, abs=1e-15)
    rng = np.random.default_rng(3)
    for nh in range(1, 5):
        wf, ws = oracle.cfm4_weights(nh)
        assert wf.sum() == pytest.approx(1.0, abs=1e-13) and ws.sum() == pytest.approx(1.0, abs=1e-13)
        xs = -np.arange(nh, dtype=float)       # history offsets, newest first
        coef = rng.standard_normal(nh)         # a random polynomial of degree nh - 1
        p = np.polynomial.polynomial.Polynomial(coef)
        assert wf @ p(xs) == pytest.approx(2 * (a2 * p(th1) + a1 * p(th2)), abs=1e-12)
        assert ws @ p(xs) == pytest.approx(2 * (a1 * p(th1) + a2 * p(th2)), abs=1e-12)


def _cfm_case(xc):
    spec = I.SystemSpec(nx=12, ny=12, nz=12, h=0.5, fd_order=4, prec=I.PREC_C128, n_orb=2, n_atoms=2,
                        projectors=False, gauge=I.GAUGE_LENGTH, amp=0.3, omega=3.0, dt=0.02, seed=9)
    inp = I.make_inputs(spec)
    return spec, inp, oracle.System(spec, inp, xc=xc)


def test_cfm4_without_field_is_two_taylor_half_steps():
    """With H time-independent (no field, no exchange) both exponentials are exp(-i dt/2 H):
    a CFM4 step is two Taylor-4 steps of dt/2."""
    spec, inp, o = _cfm_case(0)
    o0 = oracle.System(spec, inp, xc=0, gauge=I.GAUGE_NONE)
    c, obs_c = o0.propagate_cfm4(inp.psi0, 0.0, 0.04, 5, 1)
    t, obs_t = o0.propagate(inp.psi0, 0.0, 0.04, 5, 2)
    assert np.max(np.abs(c - t)) < 1e-14
    np.testing.assert_allclose(obs_c, obs_t, rtol=1e-13, atol=1e-14)


def test_cfm4_is_fourth_order_for_a_driven_linear_problem():
    """Fast laser (omega = 3 Ha), no exchange: halving dt divides the CFM4 error by 16
    (Taylor-4 with the field at the step midpoint: by 4); reference: CFM4 at dt/32."""
    spec, inp, o = _cfm_case(0)
    T = 0.64
    ref, _ = o.propagate_cfm4(inp.psi0, 0.0, T / 256, 256, 1, record=False)
    e = [np.linalg.norm(o.propagate_cfm4(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (8, 16, 32)]
    et = [np.linalg.norm(o.propagate(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (8, 16, 32)]
    for a, b in zip(e, e[1:]):
        assert 14.0 < a / b < 18.0
    for a, b in zip(et, et[1:]):
        assert 3.5 < a / b < 5.0
    assert e[-1] < 0.02 * et[-1]


def test_cfm4_with_exchange_converges_faster_than_taylor():
    """With LDA exchange v_x at the Gauss points comes from the extrapolated history; the
    first three sub-steps have fewer than four points, which lowers the observed order (~3:
    error ratio > 6 per halving) but keeps it above Taylor-4 with a frozen density (~1)."""
    spec, inp, o = _cfm_case(1)
    T = 0.64
    ref, _ = o.propagate_cfm4(inp.psi0, 0.0, T / 256, 256, 1, record=False)
    e = [np.linalg.norm(o.propagate_cfm4(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (16, 32, 64)]
    et = [np.linalg.norm(o.propagate(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (16, 32, 64)]
    for a, b in zip(e, e[1:]):
        assert a / b > 6.0
    for a, b in zip(et, et[1:]):
        assert 1.7 < a / b < 2.3


# ---------------------------------------------------------------------------------------
# Exponential midpoint rule and approximate enforced time-reversal symmetry (named among the
# propagators in use, Sec. "New propagators for real-time TDDFT"; forms as the oracle states)
# ---------------------------------------------------------------------------------------
def test_emr_and_aetrs_reduce_to_taylor_steps_without_exchange():
    """H time-independent (no field, no exchange): an EMR step is one Taylor-4 step of dt and
    an AETRS step two of dt/2.  With the field but no exchange, EMR is the Taylor-4 step with
    the field at the midpoint: the plain propagator."""
    spec, inp, o = _cfm_case(0)
    o0 = oracle.System(spec, inp, xc=0, gauge=I.GAUGE_NONE)
    e, obs_e = o0.propagate_emr(inp.psi0, 0.0, 0.04, 5, 1)
    t1, obs_t1 = o0.propagate(inp.psi0, 0.0, 0.04, 5, 1)
    a, obs_a = o0.propagate_aetrs(inp.psi0, 0.0, 0.04, 5, 1)
    t2, obs_t2 = o0.propagate(inp.psi0, 0.0, 0.04, 5, 2)
    assert np.max(np.abs(e - t1)) < 1e-14 and np.max(np.abs(a - t2)) < 1e-14
    np.testing.assert_allclose(obs_e, obs_t1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(obs_a, obs_t2, rtol=1e-13, atol=1e-14)
    ef, _ = o.propagate_emr(inp.psi0, 0.0, 0.04, 5, 1)
    tf, _ = o.propagate(inp.psi0, 0.0, 0.04, 5, 1)
    assert np.max(np.abs(ef - tf)) < 1e-14
    af, _ = o.propagate_aetrs(inp.psi0, 0.0, 0.04, 5, 1)
    assert np.max(np.abs(af - tf)) > 1e-6  # the field enters at t and t + dt instead


def _orders(o, inp, fn, T, ns):
    ref, _ = o.propagate_cfm4(inp.psi0, 0.0, T / 256, 256, 1, record=False)
    e = [np.linalg.norm(fn(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in ns]
    return [a / b for a, b in zip(e, e[1:])]


def test_aetrs_is_second_order_for_a_driven_linear_problem():
    """Fast laser, no exchange: halving dt divides the AETRS error by 4 (order two of the
    trapezoid-like split); reference: CFM4 at dt/32."""
    spec, inp, o = _cfm_case(0)
    for r in _orders(o, inp, o.propagate_aetrs, 0.64, (8, 16, 32)):
        assert 3.5 < r < 4.6, r


@pytest.mark.parametrize("name", ["emr", "aetrs"])
def test_emr_and_aetrs_with_exchange_are_second_order(name):
    """With LDA exchange, v_x at t + dt/2 (EMR) or t + dt (AETRS) comes from the extrapolated
    history: both stay order two (error ratio ~4 per halving), where Taylor-4 with the density
    frozen over the step is order one (ratio ~2)."""
    spec, inp, o = _cfm_case(1)
    for r in _orders(o, inp, getattr(o, "propagate_" + name), 0.64, (16, 32, 64)):
        assert 3.4 < r < 4.8, (name, r)


# ---------------------------------------------------------------------------------------
# Enforced time-reversal symmetry with its trial state (the scheme of the propagator review
# the paper cites beside EMR; forms as the oracle states)
# ---------------------------------------------------------------------------------------
def test_etrs_without_exchange_is_the_aetrs_step():
    """Without a density-dependent potential the trial state changes nothing: the ETRS step is
    exp(-i dt/2 H[t + dt]) exp(-i dt/2 H[t]), the AETRS step, with the field at t and t + dt."""
    spec, inp, o = _cfm_case(0)
    e, obs_e = o.propagate_etrs(inp.psi0, 0.0, 0.04, 5, 2)
    a, obs_a = o.propagate_aetrs(inp.psi0, 0.0, 0.04, 5, 2)
    assert np.max(np.abs(e - a)) == 0.0
    np.testing.assert_array_equal(obs_e, obs_a)


def _taylor4(z):
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def test_etrs_on_plane_waves_with_exchange_is_closed_form():
    """Plane waves in a cell keep a uniform density, so H acts on each as the number
    lam_j = kappa_j + v_x(n) and every exponential is the scalar Taylor polynomial R(-i tau lam).
    One ETRS sub-step: the trial multiplies plane wave j by R(-i dt lam_j) (uniform density
    n~ = sum f |amplitude|^2 / V), then phi_j <- R(-i dt/2 (kappa_j + v_x(n~))) R(-i dt/2 lam_j)
    phi_j.  A trial of dt/2, or v_x of the old density in the second half, misses by >1e-8."""
    spec, inp, psi, qs = _plane_wave_case(4, I.GAUGE_NONE)
    spec = dataclasses.replace(spec, xc=I.XC_LDA_X, amp=0.0)
    o = oracle.System(spec, inp)
    vol = spec.n_points * spec.h ** 3
    psi = psi / math.sqrt(vol)
    kap = np.array([[_pw_eigen(spec, qs[ik, j], np.zeros(3))[0] for j in range(3)] for ik in range(2)])
    dt, n_steps = 0.8 / np.max(np.abs(kap)), 3
    vx = lambda n: -(3 * n / math.pi) ** (1 / 3)
    dens = lambda amp: spec.occ * float(np.sum(inp.kw[:, None] * np.abs(amp) ** 2)) / vol

    def closed(trial_frac, use_trial):
        amp = np.ones((2, 3), dtype=complex)
        for _ in range(n_steps):
            lam1 = kap + vx(dens(amp))
            lam2 = kap + vx(dens(amp * _taylor4(-1j * trial_frac * dt * lam1))) if use_trial else lam1
            amp = amp * _taylor4(-0.5j * dt * lam1) * _taylor4(-0.5j * dt * lam2)
        return amp

    got, _ = o.propagate_etrs(psi, 0.0, dt, n_steps, 1, record=False)
    want = closed(1.0, True)
    for ik in range(2):
        for j in range(3):
            np.testing.assert_allclose(got[ik, ..., j], want[ik, j] * psi[ik, ..., j], rtol=0, atol=1e-13 / math.sqrt(vol))
    for wrong in (closed(0.5, True), closed(1.0, False)):
        assert np.max(np.abs(wrong - want)) > 1e-8


def test_etrs_with_exchange_is_second_order():
    """With LDA exchange the trial state supplies v_x at t + dt: ETRS stays order two (error
    ratio ~4 per halving; reference: CFM4 at dt/256)."""
    spec, inp, o = _cfm_case(1)
    for r in _orders(o, inp, o.propagate_etrs, 0.64, (16, 32, 64)):
        assert 3.4 < r < 4.8, r


# ---------------------------------------------------------------------------------------
# Classical Runge-Kutta 4 (Runge-Kutta is in the same section's list of propagators)
# ---------------------------------------------------------------------------------------
def test_rk4_without_field_or_exchange_is_the_taylor_step():
    """For a time-independent linear H the RK4 update is exactly the degree-4 Taylor polynomial
    of exp(-i dt H): one RK4 step equals one Taylor-4 step up to rounding."""
    spec, inp, o = _cfm_case(0)
    o0 = oracle.System(spec, inp, xc=0, gauge=I.GAUGE_NONE)
    r, obs_r = o0.propagate_rk4(inp.psi0, 0.0, 0.04, 5, 1)
    t, obs_t = o0.propagate(inp.psi0, 0.0, 0.04, 5, 1)
    assert np.max(np.abs(r - t)) < 1e-13
    np.testing.assert_allclose(obs_r, obs_t, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("xc", [0, 1])
def test_rk4_is_fourth_order_with_field_and_exchange(xc):
    """Driven problem, with and without LDA exchange: the stages rebuild the density, so the
    error falls 16x per halving of dt in both cases (reference: RK4 at dt/32)."""
    spec, inp, o = _cfm_case(xc)
    T = 0.64
    ref, _ = o.propagate_rk4(inp.psi0, 0.0, T / 256, 256, 1, record=False)
    e = [np.linalg.norm(o.propagate_rk4(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (8, 16, 32)]
    for a, b in zip(e, e[1:]):
        assert 14.0 < a / b < 18.0, e


def test_rk4_velocity_gauge_agrees_with_taylor_at_small_steps():
    """Periodic cell in the velocity gauge (H depends on A(t) non-linearly): RK4 and Taylor-4
    (exchange off, so Taylor-4 is order two through the midpoint field) converge to the same
    state; their difference falls ~4x per halving of dt."""
    from tests._util import bloch_cell, bloch_inputs
    spec = bloch_cell(I.PREC_C128)
    inp = bloch_inputs(spec)
    o = oracle.System(spec, inp, xc=0)
    T = 0.16
    d = []
    for n in (4, 8, 16):
        a, _ = o.propagate_rk4(inp.psi0, 0.0, T / n, n, 1, record=False)
        b, _ = o.propagate(inp.psi0, 0.0, T / n, n, 1, record=False)
        d.append(np.linalg.norm(a - b))
    for x, y in zip(d, d[1:]):
        assert 3.3 < x / y < 4.8, d


# ---------------------------------------------------------------------------------------
# Hartree potential (the density-dependent potential beside exchange in the TDDFT
# Hamiltonian): a direct sum over grid cells in a box, the plane-wave Poisson solve in a cell
# ---------------------------------------------------------------------------------------
def test_hartree_self_cell_constant_by_quadrature():
    """c0 = int over the unit cube of 1/|r|: adaptive cubature over one octant, times 8."""
    from scipy import integrate
    val, err = integrate.nquad(lambda x, y, z: 1.0 / math.sqrt(x * x + y * y + z * z), [[0.0, 0.5]] * 3,
                               opts={"epsabs": 1e-11, "epsrel": 1e-11, "limit": 100})
    assert oracle.hartree_self_cell() == pytest.approx(8.0 * val, abs=1e-9)


def _gaussian_box(n, h, sigma, xc=0):
    spec = _spec(nx=n, ny=n, nz=n, h=h, n_orb=1, xc=xc)
    o = oracle.System(spec, I.make_inputs(spec, with_orbitals=False))
    x = (np.arange(n) - (n - 1) / 2) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    dens = np.exp(-r * r / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2) ** 1.5
    return o, r, dens


def test_hartree_of_a_gaussian_converges_to_the_closed_form():
    """n = normalised Gaussian of width sigma: v_H = erf(r / (sqrt2 sigma)) / r and
    E_H = 1 / (2 sqrt(pi) sigma).  The cell sum is second order in h: halving h cuts the
    error of both by more than 3 (the box edge at 4 sigma limits the ratio slightly)."""
    from scipy import special
    errs, eerrs = [], []
    for n, h in ((16, 0.5), (32, 0.25)):
        o, r, dens = _gaussian_box(n, h, 1.0)
        eh, vh = o.hartree(dens.ravel())
        exact = np.where(r > 0, special.erf(r / math.sqrt(2.0)) / np.maximum(r, 1e-300), math.sqrt(2 / math.pi))
        errs.append(np.abs(vh.reshape(r.shape) - exact).max())
        eerrs.append(abs(eh - 1 / (2 * math.sqrt(math.pi))))
    assert errs[0] < 7e-3 and errs[1] < 2e-3 and errs[0] > 3.0 * errs[1], errs
    assert eerrs[0] < 1.5e-3 and eerrs[0] > 3.0 * eerrs[1], eerrs


def test_hartree_far_field_is_the_total_charge_over_r():
    """Far from a compact, cubically symmetric charge the potential is Q/r (the quadrupole
    vanishes by symmetry; the next term is (sigma/r)^4 ~ 1e-4 here)."""
    o, r, dens = _gaussian_box(21, 0.4, 0.6)
    _, vh = o.hartree(dens.ravel())
    q = dens.sum() * 0.4 ** 3
    corner = np.unravel_index(np.argmax(r), r.shape)
    assert vh.reshape(r.shape)[corner] == pytest.approx(q / r[corner], rel=1e-3)


def test_hartree_kernel_is_symmetric_and_linear():
    """<n1, v_H[n2]> = <n2, v_H[n1]> and v_H[a n1 + n2] = a v_H[n1] + v_H[n2], in a box and in a
    cell (a transposed or offset kernel breaks the first)."""
    rng = np.random.default_rng(8)
    for bc in (I.BC_ZERO, I.BC_BLOCH):
        spec = _spec(nx=7, ny=6, nz=5, h=0.4, n_orb=1, bc=bc, xc=0)
        o = oracle.System(spec, I.make_inputs(spec, with_orbitals=False))
        n1, n2 = rng.random(spec.n_points), rng.random(spec.n_points)
        v1, v2 = o.hartree(n1)[1], o.hartree(n2)[1]
        assert n1 @ v2 == pytest.approx(n2 @ v1, rel=1e-12)
        v12 = o.hartree(2.5 * n1 + n2)[1]
        np.testing.assert_allclose(v12, 2.5 * v1 + v2, rtol=1e-12, atol=1e-12 * np.abs(v12).max())


def test_hartree_of_plane_waves_in_a_cell_is_exact():
    """Periodic cell: n = cos(G.r) gives v_H = 4 pi / |G|^2 cos(G.r) (the background removes
    the mean); checked for three waves at once, one at the Nyquist index of an even axis."""
    spec = _spec(nx=6, ny=5, nz=4, h=0.4, n_orb=1, bc=I.BC_BLOCH, xc=0)
    o = oracle.System(spec, I.make_inputs(spec, with_orbitals=False))
    L = np.array([6, 5, 4]) * 0.4
    z, y, x = np.meshgrid(np.arange(4) * 0.4, np.arange(5) * 0.4, np.arange(6) * 0.4, indexing="ij")
    waves = [((2 * math.pi / L[0], 0, 0), 1.0), ((0, 4 * math.pi / L[1], 2 * math.pi / L[2]), 0.5),
             ((math.pi / 0.4, 0, 0), 0.25)]
    n = 3.0 + sum(a * np.cos(g[0] * x + g[1] * y + g[2] * z) for g, a in waves)
    want = sum(a * 4 * math.pi / (g[0] ** 2 + g[1] ** 2 + g[2] ** 2) * np.cos(g[0] * x + g[1] * y + g[2] * z)
               for g, a in waves)
    eh, vh = o.hartree(n.ravel())
    np.testing.assert_allclose(vh, want.ravel(), atol=1e-11)
    assert eh == pytest.approx(0.5 * float(n.ravel() @ vh) * 0.4 ** 3, rel=1e-12)


# Exchange and Hartree together (xc 2): the density-dependent potential v_x + v_H wherever
# the propagators rebuild or extrapolate it, and E_H in the recorded energy.
def test_hartree_enters_the_energy_as_exactly_e_h():
    """For one state, the recorded energy with Hartree minus the one without is E_H: the band
    term gains int n v_H, the double-counting correction removes it, and E_H = 1/2 int n v_H is
    added (a dropped or doubled piece breaks the equality)."""
    spec, inp, _ = _cfm_case(1)
    o1 = oracle.System(spec, inp, xc=1)
    o2 = oracle.System(spec, inp, xc=2)
    e1 = o1.observables(inp.psi0, 0.0, 0.1)
    e2 = o2.observables(inp.psi0, 0.0, 0.1)
    eh, _ = o2.hartree(o2.density(inp.psi0).ravel())
    assert eh > 0
    assert e2[2] - e1[2] == pytest.approx(eh, rel=1e-11)
    assert e2[3] == e1[3] and e2[1] == e1[1]  # E_x and the norm are unchanged


def test_hartree_energy_conservation_is_first_order_with_the_frozen_density():
    """Zero field, exchange and Hartree: Taylor-4 freezes both over a step, so the energy drift
    over a fixed time falls ~2x when dt halves, as with exchange alone."""
    spec = _spec(nx=12, ny=12, nz=12, h=0.4, fd_order=4, n_orb=2, n_atoms=2, wells=True, xc=2, seed=6)
    inp = I.make_inputs(spec)
    o = oracle.System(spec, inp, xc=2)
    drifts = []
    for dt, nst in ((0.02, 20), (0.01, 40)):
        psi_end, obs = o.propagate(inp.psi0, 0.0, dt, nst, 1)
        drifts.append(abs(o.observables(psi_end, dt * nst, dt * nst)[2] - obs[0, 2]))
    assert drifts[0] < 2e-3 * abs(obs[0, 2])
    assert 1.7 * drifts[1] < drifts[0] < 2.4 * drifts[1], drifts


def test_rk4_and_cfm4_with_hartree_keep_their_order():
    """Driven problem with exchange and Hartree: RK4 (every stage rebuilds v_x + v_H) stays
    fourth order (ratio ~16 per halving); CFM4 (v_x + v_H extrapolated from the history)
    converges faster than second order (ratio > 6)."""
    spec, inp, o = _cfm_case(2)
    T = 0.64
    ref, _ = o.propagate_rk4(inp.psi0, 0.0, T / 256, 256, 1, record=False)
    er = [np.linalg.norm(o.propagate_rk4(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (8, 16, 32)]
    ec = [np.linalg.norm(o.propagate_cfm4(inp.psi0, 0.0, T / n, n, 1, record=False)[0] - ref) for n in (16, 32, 64)]
    for a, b in zip(er, er[1:]):
        assert 14.0 < a / b < 18.0, er
    for a, b in zip(ec, ec[1:]):
        assert a / b > 6.0, ec


@pytest.mark.parametrize("name", ["emr", "aetrs", "etrs"])
def test_two_point_propagators_with_hartree_stay_second_order(name):
    """Exchange and Hartree: EMR and AETRS (v_x + v_H extrapolated from the history) and ETRS
    (v_x + v_H of the trial's density) stay order two (error ratio ~4 per halving)."""
    spec, inp, o = _cfm_case(2)
    for r in _orders(o, inp, getattr(o, "propagate_" + name), 0.64, (16, 32, 64)):
        assert 3.4 < r < 4.8, (name, r)


# Current of a periodic cell with the projectors' commutator (Sec. "Conductivities": the
# velocity operator i[H, r] includes i[V_NL, r]); the record carries both parts.
def test_current_is_minus_the_energy_derivative_in_a():
    """J = -(1/Omega) dE/dA on the discrete level, because H(A) depends on A only through
    -i A.grad_h + |A|^2/2 and the projectors' gauge phases: the velocity expectation with the
    projector commutator equals the central difference of the band energy in each component of
    A (error ~delta^2), while the local part alone misses by the projectors' share."""
    from tests._util import bloch_cell, bloch_inputs
    spec = bloch_cell(I.PREC_C128, n_k=2)
    inp = bloch_inputs(spec)
    o = oracle.System(spec, inp, xc=0)
    A = np.array([0.07, -0.05, 0.11])
    d = 1e-4
    fd = np.array([(o.band_energy(A + d * e, inp.psi0) - o.band_energy(A - d * e, inp.psi0)) / (2 * d)
                   for e in np.eye(3)])
    full, local = o.velocity(A, inp.psi0), o.velocity(A, inp.psi0, with_nonlocal=False)
    scale = np.abs(full).max()
    assert np.abs(fd - full).max() < 1e-8 * scale
    assert np.abs(fd - local).max() > 1e-2 * scale
    # without projectors the commutator vanishes
    o0 = oracle.System(spec, inp, xc=0, projectors=False)
    np.testing.assert_array_equal(o0.velocity(A, inp.psi0), o0.velocity(A, inp.psi0, with_nonlocal=False))


def test_recorded_current_is_minus_the_energy_derivative():
    """The record's current is -(1/Omega) times the full velocity expectation at A(t_field),
    projectors' commutator included, so it equals -(1/Omega) dE/dA by central differences."""
    from tests._util import bloch_cell, bloch_inputs
    spec = bloch_cell(I.PREC_C128, n_k=2)
    inp = bloch_inputs(spec)
    o = oracle.System(spec, inp, xc=0)
    obs = o.observables(inp.psi0, 0.0, 0.3)
    _, A = o.field(0.3)
    omega = spec.nx * spec.ny * spec.nz * spec.h ** 3
    np.testing.assert_allclose(obs[4:7], -o.velocity(A, inp.psi0) / omega, rtol=1e-12, atol=1e-14)
    d = 1e-4
    fd = np.array([(o.band_energy(A + d * e, inp.psi0) - o.band_energy(A - d * e, inp.psi0)) / (2 * d)
                   for e in np.eye(3)])
    assert np.abs(obs[4:7] + fd / omega).max() < 1e-8 * np.abs(fd / omega).max()


def test_hartree_cell_sum_equals_a_zero_padded_fft_convolution():
    """The box's cell sum is a linear convolution with the sampled kernel (1/|d|, c0/h at
    d = 0), so a zero-padded FFT convolution (Hockney) reproduces it to rounding: the method a
    GPU kernel can use, checked here with numpy's FFT on a random density."""
    spec = _spec(nx=9, ny=8, nz=7, h=0.3, n_orb=1, xc=0)
    o = oracle.System(spec, I.make_inputs(spec, with_orbitals=False))
    rng = np.random.default_rng(21)
    n = rng.random((spec.nz, spec.ny, spec.nx))
    shape = (2 * spec.nz, 2 * spec.ny, 2 * spec.nx)
    idx = [np.where(np.arange(m) < m // 2, np.arange(m), np.arange(m) - m) for m in shape]
    dz, dy, dx = np.meshgrid(*idx, indexing="ij")
    dist = spec.h * np.sqrt(dx * dx + dy * dy + dz * dz)
    kern = np.where(dist > 0, 1.0 / np.where(dist > 0, dist, 1.0), oracle.hartree_self_cell() / spec.h)
    # offsets of magnitude n along an axis never occur inside the box; keep them out of the wrap
    for ax, m in enumerate(shape):
        sl = [slice(None)] * 3
        sl[ax] = m // 2
        kern[tuple(sl)] = 0.0
    pad = np.zeros(shape)
    pad[:spec.nz, :spec.ny, :spec.nx] = n
    conv = np.fft.irfftn(np.fft.rfftn(pad) * np.fft.rfftn(kern), s=shape, axes=(0, 1, 2))[:spec.nz, :spec.ny, :spec.nx]
    _, vh = o.hartree(n.ravel())
    np.testing.assert_allclose(vh, conv.ravel() * spec.h ** 3, rtol=1e-12, atol=1e-12 * np.abs(vh).max())


def test_energy_with_projectors_and_length_gauge_field_is_the_dense_expectation():
    """The recorded energy of a finite box with projectors, wells, LDA exchange and a
    length-gauge field, against sum_i f <phi_i|H0|phi_i> h^3 + E_x built here densely: the
    kinetic matrix from the golden FD weights, the wells, +E(t).r with E written out, and the
    brute-force projector matrix (the exchange terms of the record cancel except E_x, which
    is the Dirac expression of the density formed here)."""
    spec = _spec(nx=8, ny=8, nz=8, h=0.45, fd_order=4, n_orb=2, n_atoms=2, projectors=True, wells=True,
                 xc=I.XC_LDA_X, gauge=I.GAUGE_LENGTH, amp=0.3, omega=0.7, pol=(0.3, -0.5, 0.8), seed=5)
    inp = I.make_inputs(spec)
    o = oracle.System(spec, inp)
    psi = I.random_orbitals(spec, 31) * 0.3
    t_field = 1.1
    rec = o.observables(psi, 0.0, t_field)
    n = spec.n_points
    h = spec.h
    c = [float(v) for v in _read_golden()[("lap", 4)]]
    x = _axis(spec, spec.nx)
    D1 = np.zeros((spec.nx, spec.nx))
    for i in range(spec.nx):
        D1[i, i] = c[0]
        for m in (1, 2):
            if i + m < spec.nx:
                D1[i, i + m] = D1[i + m, i] = c[m]
    I1 = np.eye(spec.nx)
    lap = (np.kron(np.kron(D1, I1), I1) + np.kron(np.kron(I1, D1), I1) + np.kron(np.kron(I1, I1), D1)) / h ** 2
    E = spec.amp * math.sin(spec.omega * t_field) * np.array(spec.pol)
    X, Y, Z = _grids(spec)
    er = (E[0] * X + E[1] * Y + E[2] * Z).reshape(-1)
    H0 = -0.5 * lap + np.diag(inp.vloc.reshape(-1) + er) + _dense_vnl(spec, inp, np.zeros(3), np.zeros(3))
    band = sum(spec.occ * np.vdot(psi[0, ..., j].reshape(-1), H0 @ psi[0, ..., j].reshape(-1)).real * h ** 3
               for j in range(spec.n_orb))
    dens = spec.occ * np.sum(np.abs(psi[0]) ** 2, axis=-1)
    ex = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * np.sum(dens ** (4.0 / 3.0)) * h ** 3
    assert rec[3] == pytest.approx(ex, rel=1e-12)
    assert rec[2] == pytest.approx(band + ex, rel=1e-12)
    assert rec[7] == pytest.approx(E @ np.array(spec.pol), rel=1e-12)


# Kinetic heat current (Sec. "Conductivities", eqn. KEcurrent; the reading with the last pair
# antisymmetric, covariant derivatives).  On a periodic grid every discrete operator in it is
# diagonal in the grid's plane waves q = k + 2 pi n / L: the covariant gradient has the symbol
# i kappa = i (qd + A) (qd the central difference's symbol), the covariant Laplacian -Lambda =
# -(lambda + 2 A.qd + |A|^2) (lambda the star Laplacian's), the composed second differences
# -kappa_i kappa_j.  So J_t = sum_k w_k f sum_q |a_q|^2 (-1/4) kappa_q (Lambda_q + |kappa_q|^2), with
# a_q the state's plane-wave amplitudes (numpy's FFT), and for a plane wave in the continuum limit
# -(1/2)|k|^2 k: minus its kinetic energy times its velocity.
def _heat_symbols(spec, q, A):
    M = spec.fd_order // 2
    c, d = oracle.fd_weights(M)
    h = spec.h
    qd = np.array([2.0 / h * sum(d[m] * math.sin(m * qa * h) for m in range(1, M + 1)) for qa in q])
    lam = sum((-c[0] - 2 * sum(c[m] * math.cos(m * qa * h) for m in range(1, M + 1))) / (h * h) for qa in q)
    kappa = qd + A
    Lam = lam + 2.0 * A @ qd + A @ A
    return -0.25 * kappa * (Lam + kappa @ kappa)


@pytest.mark.parametrize("fd_order", [4, 8])
def test_heat_current_of_plane_waves(fd_order):
    spec, inp, psi, qs = _plane_wave_case(fd_order, I.GAUGE_VELOCITY)
    o = oracle.System(spec, inp)
    A = np.array([0.07, -0.12, 0.2])
    got = o.heat_current(A, psi)
    want = sum(inp.kw[ik] * spec.occ * _heat_symbols(spec, qs[ik, j], A) for ik in range(2) for j in range(3))
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13 * np.abs(want).max())
    # continuum limit of one plane wave: minus its kinetic energy times its velocity
    spec1 = dataclasses.replace(spec, h=0.01)
    q = np.array([0.3, -0.2, 0.5])
    np.testing.assert_allclose(_heat_symbols(spec1, q, np.zeros(3)), -0.5 * (q @ q) * q, rtol=1e-4)


def test_heat_current_of_random_bloch_states_is_diagonal_in_plane_waves():
    spec = _spec(nx=8, ny=6, nz=5, h=0.4, fd_order=4, bc=I.BC_BLOCH, n_orb=2, n_k=2, seed=9)
    inp = _inputs(spec)
    o = oracle.System(spec, inp)
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    X, Y, Z = _grids(spec)
    rng = np.random.Generator(np.random.PCG64(7))
    A = np.array([0.15, 0.05, -0.1])
    psi = np.empty((2, spec.nz, spec.ny, spec.nx, 2), dtype=np.complex128)
    want = np.zeros(3)
    for ik in range(2):
        k = inp.kpts[ik]
        for j in range(2):
            u = rng.standard_normal((spec.nz, spec.ny, spec.nx)) + 1j * rng.standard_normal((spec.nz, spec.ny, spec.nx))
            psi[ik, ..., j] = np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z)) * u
            a = np.fft.fftn(u) / u.size  # u = sum_n a_n exp(2 pi i n.r / L)
            for (nz_, ny_, nx_), amp in np.ndenumerate(a):
                n = np.array([nx_ if nx_ <= spec.nx // 2 else nx_ - spec.nx,
                              ny_ if ny_ <= spec.ny // 2 else ny_ - spec.ny,
                              nz_ if nz_ <= spec.nz // 2 else nz_ - spec.nz])
                want += inp.kw[ik] * spec.occ * abs(amp) ** 2 * _heat_symbols(spec, k + 2 * np.pi * n / L, A)
    got = o.heat_current(A, psi)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
