"""The seeded input generator shared by the library's tests and the oracle: SplitMix64 against
its published reference outputs (tests/golden/splitmix64.txt), orthonormal initial orbitals
(h^3 inner product), the Bloch condition of periodic orbitals, k-points in the first zone, and
determinism of every workload's inputs."""
import os

import numpy as np

from paper_1912_07921_gb300 import inputs as I


def test_splitmix64_reference_outputs():
    lines = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    want = [int(l[0]) for l in lines[1:]]
    g = I.SplitMix64(seed)
    assert [g.next_u64() for _ in want] == want


def test_initial_orbitals_are_orthonormal_in_a_box_and_a_cell():
    for spec in (I.SystemSpec(nx=14, ny=12, nz=10, h=0.35, n_orb=5, seed=3),
                 I.SystemSpec(nx=10, ny=9, nz=8, h=0.4, n_orb=4, n_k=3, bc=I.BC_BLOCH, seed=4)):
        psi = I.initial_orbitals(spec)
        for k in range(psi.shape[0]):
            a = psi[k].reshape(-1, spec.n_orb)
            np.testing.assert_allclose(a.conj().T @ a * spec.h ** 3, np.eye(spec.n_orb), atol=1e-12)


def test_periodic_orbitals_are_bloch_states_smooth_across_the_faces():
    """The orbitals are exp(i k.r) times a periodic envelope built from the nearest Gaussian
    images, so with the Bloch condition psi(r + L e_x) = exp(i k_x L) psi(r) the envelope is as
    smooth across the x face as between interior neighbours; k lies in the first zone."""
    spec = I.SystemSpec(nx=12, ny=6, nz=5, h=0.4, n_orb=2, n_k=2, bc=I.BC_BLOCH, seed=9)
    psi = I.initial_orbitals(spec)
    k, _ = I.kpoints(spec)
    x = np.arange(spec.nx) * spec.h
    for ik in range(k.shape[0]):
        env = psi[ik] * np.exp(-1j * k[ik, 0] * x)[None, None, :, None]
        jump = np.abs(env[:, :, 0] - env[:, :, -1]).max()   # across the face
        step = np.abs(np.diff(env, axis=2)).max()            # largest interior step
        assert jump <= 1.01 * step
        assert np.all(np.abs(k[ik]) <= np.pi / (np.array([spec.nx, spec.ny, spec.nz]) * spec.h))


def test_workload_inputs_are_deterministic():
    for spec in (I.tiny_molecule(), I.SystemSpec(nx=10, ny=9, nz=8, h=0.4, n_orb=3, n_atoms=2, projectors=True,
                                                 bc=I.BC_BLOCH, n_k=2, seed=5)):
        a, b = I.make_inputs(spec), I.make_inputs(spec)
        for f in ("vloc", "psi0", "pos", "D", "kpts", "kw"):
            np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
