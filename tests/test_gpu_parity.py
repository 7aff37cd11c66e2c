"""CUDA path against the FP64 oracle, through the C interface, on the same seeded inputs.

Tolerances: complex128 systems match the oracle to 1e-12 relative (max-norm over all
values); complex64 systems run H psi in FP32, where a 25-point stencil sum of values of
size |psi| carries a relative rounding error of ~1e-7 * (sum |c_m| / |c_0|) < 1e-6 of the
largest value, so single H applications are checked to 5e-6 and the dipole over 1000
steps to 1e-4 of its peak.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I
from tests._util import bloch_cell, bloch_inputs, ragged_molecule, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _system(spec, inp, **kw):
    from paper_1912_07921_gb300.system import System
    return System(spec, inp, stream=torch.cuda.current_stream().cuda_stream, **kw)


def _apply_gpu(sysm, psi, t):
    packed = sysm.pack(psi)
    din = torch.from_numpy(packed.view(np.float32 if packed.dtype == np.complex64 else np.float64)).cuda()
    dout = torch.empty_like(din)
    sysm.apply_H(t, din.data_ptr(), dout.data_ptr())
    torch.cuda.synchronize()
    out = dout.cpu().numpy().view(packed.dtype).reshape(packed.shape)
    return sysm.unpack(out)


def _minimal_box(prec):
    """5^3 finite box at order 8 (M + 1 points per axis), one orbital, one atom whose
    projector sphere covers the whole box."""
    return I.SystemSpec(nx=5, ny=5, nz=5, h=0.4, fd_order=8, prec=prec, n_orb=1, n_atoms=1, projectors=True,
                        gauge=I.GAUGE_LENGTH, amp=0.05, omega=0.3, dt=0.005, seed=12)


def _minimal_cell(prec):
    """2^3 periodic cell at order 4 (M points per axis): every halo point is a periodic image
    of the cell itself, with its Bloch phase."""
    return bloch_cell(prec, nx=2, ny=2, nz=2, n_orb=2, n_k=2)


APPLY_CASES = {
    "tiny_c128": (lambda: I.tiny_molecule(), None),
    "ragged_c128_order8": (lambda: ragged_molecule(I.PREC_C128), None),
    "ragged_c128_order4": (lambda: ragged_molecule(I.PREC_C128, fd_order=4, n_orb=6), None),
    "ragged_c64_order8": (lambda: ragged_molecule(I.PREC_C64, n_orb=11), None),
    "bloch_c128_order4": (lambda: bloch_cell(I.PREC_C128), bloch_inputs),
    "bloch_c128_order8": (lambda: bloch_cell(I.PREC_C128, fd_order=8, n_k=2), bloch_inputs),
    "bloch_c64_order4": (lambda: bloch_cell(I.PREC_C64, n_orb=5), bloch_inputs),
    # degenerate sizes: the smallest grids the stencils allow, one orbital in a padded batch
    "minimal_box_c128_order8": (lambda: _minimal_box(I.PREC_C128), None),
    "minimal_box_c64_order8": (lambda: _minimal_box(I.PREC_C64), None),
    "minimal_cell_c128_order4": (lambda: _minimal_cell(I.PREC_C128), bloch_inputs),
    "minimal_cell_c64_order4": (lambda: _minimal_cell(I.PREC_C64), bloch_inputs),
}


@pytest.mark.parametrize("name", sorted(APPLY_CASES))
def test_apply_H_matches_oracle(name):
    make_spec, make_inp = APPLY_CASES[name]
    spec = make_spec()
    inp = (make_inp or I.make_inputs)(spec)
    sysm = _system(spec, inp)
    o = oracle.System(spec, inp)
    psi = I.random_orbitals(spec, 77)
    if spec.prec == I.PREC_C64:
        psi = psi.astype(np.complex64).astype(np.complex128)
    t = 0.37
    got = _apply_gpu(sysm, psi, t)
    ref = o.apply_H(psi, t, o.vx_of(inp.psi0))
    tol = 1e-12 if spec.prec == I.PREC_C128 else 5e-6
    assert rel_err(got, ref) < tol, rel_err(got, ref)
    sysm.close()


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_apply_H_is_independent_of_tile_and_sweep_path(prec):
    """TMA sweeps (warp-specialised and lockstep, 16x8 tiles) and the general sweep (any
    tile, any z-chunk) agree to the last bits of rounding (the same per-point arithmetic;
    only FMA contraction may differ)."""
    spec = ragged_molecule(prec)
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    psi = I.random_orbitals(spec, 5)
    outs = []
    for tx, ty, zc, path in ((16, 8, 0, 0), (16, 8, 0, 1), (32, 4, 0, 1), (8, 8, 5, 1), (16, 8, 7, 0), (16, 8, 7, 2),
                             (16, 8, 0, 2)):
        sysm.set_tile(tx, ty, zc)
        sysm.set_sweep_path(path)
        outs.append(_apply_gpu(sysm, psi, 0.2))
    tol = 1e-14 if prec == I.PREC_C128 else 1e-6
    for o in outs[1:]:
        assert rel_err(o, outs[0]) < tol
    sysm.close()


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_propagation_tma_and_general_paths_agree(prec):
    spec = ragged_molecule(prec)
    inp = I.make_inputs(spec)
    res = []
    for path in (0, 1, 2):
        sysm = _system(spec, inp)
        sysm.set_sweep_path(path)
        sysm.propagate(0.0, 0.02, 3, 1)
        res.append((sysm.get_orbitals(), sysm.reductions(0, 3)))
        sysm.close()
    tol = 1e-13 if prec == I.PREC_C128 else 1e-6
    for r in res[1:]:
        assert rel_err(r[0], res[0][0]) < tol
        assert rel_err(r[1], res[0][1]) < tol


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_apply_H_is_independent_of_sweep_shape(prec):
    """Every tile shape of the warp-specialised TMA sweep (16x8, 16x12 and 14x8 tiles; 1 to
    4 points per thread; 6 to 16 consumer warps) applies the same per-point arithmetic in
    the same order, on a 37 x 21 x 19 grid that is ragged for all of them."""
    from paper_1912_07921_gb300.system import shape_count, shape_info
    spec = ragged_molecule(prec, n_orb=11 if prec == I.PREC_C64 else 5)
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    psi = I.random_orbitals(spec, 9)
    outs = []
    n = shape_count()
    assert n >= 2
    for sh in range(n):
        tx, ty, rows, warps = shape_info(sh)
        vectors = 8 if sh == 5 else 4  # shape 5: one complex64 value per thread vector
        assert vectors * tx * ty == 32 * warps * rows and ty % rows == 0
        sysm.set_sweep_shape(-1, sh)
        assert sysm.sweep_shapes() == [sh] * 4
        outs.append(_apply_gpu(sysm, psi, 0.3))
    tol = 1e-14 if prec == I.PREC_C128 else 1e-6
    for o in outs[1:]:
        assert rel_err(o, outs[0]) < tol
    sysm.close()


@pytest.mark.parametrize("order", [4, 8])
def test_single_complex_shape_matches_oracle_c64(order):
    """Shape 5 (one complex64 value per thread vector, four y-adjacent points per thread) on a
    grid that is ragged for its 16 x 12 tile: H applications and a propagation with
    projectors, laser and LDA against the FP64 oracle."""
    spec = ragged_molecule(I.PREC_C64, fd_order=order, n_orb=13)
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    sysm.set_sweep_shape(-1, 5)
    psi = I.random_orbitals(spec, 21).astype(np.complex64).astype(np.complex128)
    got = _apply_gpu(sysm, psi, 0.4)
    o = oracle.System(spec, inp)
    ref = o.apply_H(psi, 0.4, o.vx_of(inp.psi0))
    assert rel_err(got, ref) < 5e-6
    sysm.propagate(0.0, 0.02, 3, 1)
    rec = sysm.reductions(0, 3)
    out = sysm.get_orbitals()
    sysm.close()
    psi_o, rec_o = o.propagate(inp.psi0, 0.0, 0.02, 3, 1)
    assert rel_err(out, psi_o) < 1e-5
    assert np.max(np.abs(rec[:, 4:7] - rec_o[:, 4:7])) < 1e-5 * np.max(np.abs(rec_o[:, 4:7]))


def test_mixed_sweep_shapes_match_oracle_c128():
    """A different tile shape for each of the four Taylor-term sweeps: the propagation
    (2 sub-steps per step, projectors, laser, LDA) still matches the FP64 oracle."""
    from paper_1912_07921_gb300.system import shape_count
    spec = ragged_molecule(I.PREC_C128)
    inp = I.make_inputs(spec)
    n = shape_count()
    sysm = _system(spec, inp)
    for sweep in range(4):
        sysm.set_sweep_shape(sweep, (sweep + 1) % n)
    sysm.propagate(0.0, 0.03, 3, 2)
    rec = sysm.reductions(0, 3)
    psi = sysm.get_orbitals()
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = o.propagate(inp.psi0, 0.0, 0.03, 3, 2)
    assert rel_err(psi, psi_o) < 1e-12
    assert _rec_err(rec, rec_o) < 1e-12


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_autotune_keeps_state_and_results(prec):
    """The autotuner times every shape on every sweep, keeps the fastest, leaves the state
    untouched, and the propagation that follows equals one with the default shapes."""
    from paper_1912_07921_gb300.system import shape_count
    spec = ragged_molecule(prec, n_orb=11 if prec == I.PREC_C64 else 5)
    inp = I.make_inputs(spec)
    a = _system(spec, inp)
    before = a.get_orbitals()
    ms = a.autotune(reps=2)
    assert ms.shape == (shape_count(), 4)
    assert np.all(ms > 0)
    assert a.sweep_shapes() == [int(i) for i in np.argmin(ms, axis=0)]
    assert np.array_equal(a.get_orbitals(), before)
    a.propagate(0.0, 0.03, 2, 2)
    b = _system(spec, inp)
    b.propagate(0.0, 0.03, 2, 2)
    tol = 1e-13 if prec == I.PREC_C128 else 1e-6
    assert rel_err(a.get_orbitals(), b.get_orbitals()) < tol
    assert rel_err(a.reductions(0, 2), b.reductions(0, 2)) < tol
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_periodic_cell_tma_sweep_matches_general_sweep(prec):
    """Bloch cells on the TMA sweep (wrapped z planes with their phase in the register
    queue, x/y neighbours across a face read with the phase, velocity-gauge gradient and
    current) agree with the general sweep, in every tile shape: H applications, and a short
    propagation with its energy and current records."""
    from paper_1912_07921_gb300.system import shape_count
    spec = bloch_cell(prec, n_orb=11 if prec == I.PREC_C64 else 5, n_k=2)
    inp = bloch_inputs(spec)
    psi = I.random_orbitals(spec, 4)
    tol = 1e-13 if prec == I.PREC_C128 else 1e-6
    ref_sys = _system(spec, inp)
    ref_sys.set_sweep_path(1)
    ref = _apply_gpu(ref_sys, psi, 0.3)
    ref_sys.propagate(0.0, 0.01, 3, 2)
    ref_psi, ref_rec = ref_sys.get_orbitals(), ref_sys.reductions(0, 3)
    ref_sys.close()
    for sh in range(shape_count()):
        sysm = _system(spec, inp)
        sysm.set_sweep_shape(-1, sh)
        assert rel_err(_apply_gpu(sysm, psi, 0.3), ref) < tol
        sysm.propagate(0.0, 0.01, 3, 2)
        assert rel_err(sysm.get_orbitals(), ref_psi) < tol
        assert rel_err(sysm.reductions(0, 3), ref_rec) < tol
        sysm.close()


def test_autotune_periodic_cell_keeps_state_and_results():
    """Periodic cells take the TMA sweep too: the autotuner times every shape, leaves the
    state untouched, and the propagation that follows matches the oracle."""
    from paper_1912_07921_gb300.system import shape_count
    spec = bloch_cell(I.PREC_C128)
    inp = bloch_inputs(spec)
    sysm = _system(spec, inp)
    before = sysm.get_orbitals()
    ms = sysm.autotune(reps=1)
    assert ms.shape == (shape_count(), 4) and np.all(ms > 0)
    assert np.array_equal(sysm.get_orbitals(), before)
    sysm.propagate(0.0, 0.03, 2, 2)
    psi, rec = sysm.get_orbitals(), sysm.reductions(0, 2)
    sysm.close()
    psi_o, rec_o = oracle.System(spec, inp).propagate(inp.psi0, 0.0, 0.03, 2, 2)
    assert rel_err(psi, psi_o) < 1e-12
    assert _rec_err(rec, rec_o) < 1e-12


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_upload_issued_during_a_propagation_is_ordered(prec):
    """tdks_set_orbitals issued right after an asynchronous tdks_propagate_n (its copy
    overlaps the propagation) replaces the state only after the propagation: the records
    equal those of an undisturbed run, and the new state is the uploaded one."""
    spec = I.tiny_molecule(prec=prec)
    inp = I.make_inputs(spec)
    a = _system(spec, inp)
    a.propagate(0.0, spec.dt, 40, 1)          # ~40 steps of GPU work still queued
    psi1 = I.random_orbitals(spec, 3)
    a.set_orbitals(psi1)                       # copied while the steps run
    rec = a.reductions(0, 40)
    got = a.get_orbitals()
    b = _system(spec, inp)
    b.propagate(0.0, spec.dt, 40, 1)
    rec_b = b.reductions(0, 40)
    assert np.array_equal(rec, rec_b)
    assert rel_err(got, psi1) < 1e-13
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["tiny_c128", "ragged_c128", "tiny_c64"])
def test_cfm4_matches_oracle(case):
    """CFM4 on the GPU (two Taylor-4 exponentials of dt/2 per sub-step with effective fields,
    the exchange potential extrapolated from the last four sub-steps) against the oracle's
    CFM4: the LDA history fills during the run; with projectors and two sub-steps per step."""
    if case == "ragged_c128":
        spec = ragged_molecule(I.PREC_C128)
        n_steps, subs, dt = 4, 2, 0.03
    else:
        spec = I.tiny_molecule(prec=I.PREC_C128 if case == "tiny_c128" else I.PREC_C64)
        n_steps, subs, dt = 12, 1, spec.dt
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    sysm.set_propagator(1)
    sysm.propagate(0.0, dt, n_steps, subs)
    psi, rec = sysm.get_orbitals(), sysm.reductions(0, n_steps)
    sysm.close()
    psi_o, rec_o = oracle.System(spec, inp).propagate_cfm4(inp.psi0, 0.0, dt, n_steps, subs)
    tol = 1e-12 if spec.prec == I.PREC_C128 else 2e-5
    assert rel_err(psi, psi_o) < tol
    assert _rec_err(rec, rec_o) < tol


@pytest.mark.parametrize("prop", ["emr", "aetrs"])
@pytest.mark.parametrize("case", ["tiny_c128", "ragged_c128", "tiny_c64"])
def test_emr_and_aetrs_match_oracle(prop, case):
    """EMR (one Taylor-4 exponential per sub-step, v_x extrapolated to the midpoint) and AETRS
    (exponentials of dt/2 with H at t, then at t + dt with v_x extrapolated there) on the GPU
    against the oracle's, as for CFM4."""
    if case == "ragged_c128":
        spec = ragged_molecule(I.PREC_C128)
        n_steps, subs, dt = 4, 2, 0.03
    else:
        spec = I.tiny_molecule(prec=I.PREC_C128 if case == "tiny_c128" else I.PREC_C64)
        n_steps, subs, dt = 12, 1, spec.dt
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    sysm.set_propagator({"emr": 2, "aetrs": 3}[prop])
    sysm.propagate(0.0, dt, n_steps, subs)
    psi, rec = sysm.get_orbitals(), sysm.reductions(0, n_steps)
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = getattr(o, "propagate_" + prop)(inp.psi0, 0.0, dt, n_steps, subs)
    tol = 1e-12 if spec.prec == I.PREC_C128 else 2e-5
    assert rel_err(psi, psi_o) < tol
    assert _rec_err(rec, rec_o) < tol


@pytest.mark.parametrize("case", ["tiny_c128", "ragged_c128", "tiny_c64", "ragged_c128_no_xc"])
def test_etrs_matches_oracle(case):
    """ETRS with its trial state (three Taylor-4 exponentials per sub-step, v_x at t + dt from
    the trial's density) on the GPU against the oracle's; without exchange it is the AETRS step."""
    if case.startswith("ragged"):
        spec = ragged_molecule(I.PREC_C128)
        n_steps, subs, dt = 4, 2, 0.03
    else:
        spec = I.tiny_molecule(prec=I.PREC_C128 if case == "tiny_c128" else I.PREC_C64)
        n_steps, subs, dt = 12, 1, spec.dt
    if case.endswith("no_xc"):
        spec = dataclasses.replace(spec, xc=I.XC_NONE)
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    sysm.set_propagator(5)
    sysm.propagate(0.0, dt, n_steps, subs)
    psi, rec = sysm.get_orbitals(), sysm.reductions(0, n_steps)
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = o.propagate_etrs(inp.psi0, 0.0, dt, n_steps, subs)
    tol = 1e-12 if spec.prec == I.PREC_C128 else 2e-5
    assert rel_err(psi, psi_o) < tol
    assert _rec_err(rec, rec_o) < tol


@pytest.mark.parametrize("case", ["ragged", "bloch"])
def test_rk4_matches_oracle(case):
    """Classical RK4 on the GPU (density rebuilt at every stage, field at the stage times)
    against the oracle's: a finite box in the length gauge with projectors and exchange, and a
    periodic cell in the velocity gauge with Bloch phases and k-points."""
    if case == "ragged":
        spec = ragged_molecule(I.PREC_C128)
        inp = I.make_inputs(spec)
        n_steps, subs, dt = 3, 2, 0.03
    else:
        spec = bloch_cell(I.PREC_C128)
        inp = bloch_inputs(spec)
        n_steps, subs, dt = 3, 2, 0.02
    sysm = _system(spec, inp)
    sysm.set_propagator(4)
    sysm.propagate(0.0, dt, n_steps, subs)
    psi, rec = sysm.get_orbitals(), sysm.reductions(0, n_steps)
    sysm.close()
    psi_o, rec_o = oracle.System(spec, inp).propagate_rk4(inp.psi0, 0.0, dt, n_steps, subs)
    assert rel_err(psi, psi_o) < 1e-12
    assert _rec_err(rec, rec_o) < 1e-12


def test_rk4_refuses_complex64():
    from paper_1912_07921_gb300 import _lib
    spec = I.tiny_molecule(prec=I.PREC_C64)
    sysm = _system(spec, I.make_inputs(spec))
    with pytest.raises(_lib.TdksError):
        sysm.set_propagator(4)
    sysm.close()


@pytest.mark.parametrize("kind", ["box", "cell"])
@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_minimal_grids_propagate_like_the_oracle(kind, prec):
    """Propagation with records on the smallest grids (see APPLY_CASES)."""
    spec = _minimal_box(prec) if kind == "box" else _minimal_cell(prec)
    inp = I.make_inputs(spec) if kind == "box" else bloch_inputs(spec)
    n_steps, subs = 3, 2
    sysm = _system(spec, inp)
    sysm.propagate(0.0, spec.dt, n_steps, subs)
    psi, rec = sysm.get_orbitals(), sysm.reductions(0, n_steps)
    sysm.close()
    psi_o, rec_o = oracle.System(spec, inp).propagate(inp.psi0, 0.0, spec.dt, n_steps, subs)
    tol = 1e-12 if prec == I.PREC_C128 else 2e-5
    assert rel_err(psi, psi_o) < tol
    assert _rec_err(rec, rec_o) < tol


def test_cfm4_refuses_the_velocity_gauge_and_batches():
    from paper_1912_07921_gb300 import _lib
    from paper_1912_07921_gb300.system import Batch
    spec = bloch_cell(I.PREC_C64)
    sysm = _system(spec, bloch_inputs(spec))
    for prop in (1, 2, 3, 5):
        sysm.set_propagator(prop)
        with pytest.raises(_lib.TdksError):
            sysm.propagate(0.0, 0.01, 1, 1)
    with pytest.raises(_lib.TdksError):
        sysm.set_propagator(6)
    sysm.close()
    spec = I.tiny_molecule(prec=I.PREC_C64)
    a = _system(spec, I.make_inputs(spec))
    a.set_propagator(1)
    a.set_clock(0.0, spec.dt, 1)
    with pytest.raises(_lib.TdksError):
        Batch([a], stream=torch.cuda.current_stream().cuda_stream)
    a.close()


def _propagate_both(spec, inp, n_steps, substeps, dt=None):
    dt = spec.dt if dt is None else dt
    sysm = _system(spec, inp)
    sysm.propagate(0.0, dt, n_steps, substeps)
    rec = sysm.reductions(0, n_steps)
    psi = sysm.get_orbitals()
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = o.propagate(inp.psi0, 0.0, dt, n_steps, substeps)
    return psi, rec, psi_o, rec_o


def _rec_err(rec, rec_o):
    """Per-column error relative to each column's scale (the dipole crosses zero)."""
    return max(float(np.max(np.abs(rec[:, c] - rec_o[:, c])) / max(np.max(np.abs(rec_o[:, c])), 1e-300))
               for c in range(rec.shape[1]) if np.max(np.abs(rec_o[:, c])) > 0)


def test_tiny_molecule_full_run_c128():
    """Tiny molecule: 24^3, order 4, 4 orbitals, 2 wells, LDA, E0=0.01, 100 steps dt=0.02."""
    spec = I.tiny_molecule()
    inp = I.make_inputs(spec)
    psi, rec, psi_o, rec_o = _propagate_both(spec, inp, spec.n_steps, spec.substeps)
    assert rel_err(psi, psi_o) < 1e-12
    assert _rec_err(rec, rec_o) < 1e-12


@pytest.mark.parametrize("case", ["ragged_c128", "bloch_c128"])
def test_short_runs_with_substeps_c128(case):
    if case == "ragged_c128":
        spec = ragged_molecule(I.PREC_C128)
        inp = I.make_inputs(spec)
    else:
        spec = bloch_cell(I.PREC_C128)
        inp = bloch_inputs(spec)
    psi, rec, psi_o, rec_o = _propagate_both(spec, inp, 4, 2, dt=0.03)
    assert rel_err(psi, psi_o) < 1e-12
    assert _rec_err(rec, rec_o) < 1e-12


def test_tiny_molecule_c64_dipole_over_1000_steps():
    """complex64 H psi with FP64 state and reductions: dipole within 1e-4 of its peak
    after 1000 steps (norm and energy checked too)."""
    spec = I.tiny_molecule(prec=I.PREC_C64, n_steps=1000)
    inp = I.make_inputs(spec)
    psi, rec, psi_o, rec_o = _propagate_both(spec, inp, spec.n_steps, spec.substeps)
    d, d_o = rec[:, 4:7], rec_o[:, 4:7]
    assert float(np.max(np.abs(d - d_o)) / np.max(np.abs(d_o))) < 1e-4
    assert float(np.max(np.abs(rec[:, 1] - rec_o[:, 1]))) < 1e-5 * rec_o[0, 1]
    assert float(np.max(np.abs(rec[:, 2] - rec_o[:, 2]))) < 1e-4 * np.max(np.abs(rec_o[:, 2]))


def test_medium_molecule_full_size_one_step_c128():
    """Medium molecule at full size (96^3, order 8, 64 orbitals, 16 atoms with projectors,
    sin^2 pulse): one configured step of 4 Taylor sub-steps, every value compared."""
    spec = I.medium_molecule(prec=I.PREC_C128)
    inp = I.make_inputs(spec)
    t0 = 20.0  # inside the pulse
    sysm = _system(spec, inp)
    sysm.propagate(t0, spec.dt, 1, spec.substeps)
    rec = sysm.reductions(0, 1)
    psi = sysm.get_orbitals()
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = o.propagate(inp.psi0, t0, spec.dt, 1, spec.substeps)
    assert rel_err(psi, psi_o) < 1e-12
    np.testing.assert_allclose(rec, rec_o, rtol=1e-12, atol=1e-12 * np.abs(rec_o).max())


def test_medium_molecule_full_size_one_step_c64():
    """Same step in the benchmark's precision (complex64 terms, FP64 state and sums)."""
    spec = I.medium_molecule(prec=I.PREC_C64)
    inp = I.make_inputs(spec)
    t0 = 20.0
    sysm = _system(spec, inp)
    assert sysm.auto_substeps(spec.dt) == spec.substeps
    sysm.propagate(t0, spec.dt, 1, spec.substeps)
    rec = sysm.reductions(0, 1)
    psi = sysm.get_orbitals()
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = o.propagate(inp.psi0, t0, spec.dt, 1, spec.substeps)
    assert rel_err(psi, psi_o) < 1e-5
    assert abs(rec[0, 1] - rec_o[0, 1]) < 1e-6 * rec_o[0, 1]
    assert abs(rec[0, 2] - rec_o[0, 2]) < 1e-5 * abs(rec_o[0, 2])
    assert np.max(np.abs(rec[0, 4:7] - rec_o[0, 4:7])) < 1e-5 * np.max(np.abs(rec_o[0, 4:7]))


def test_observe_matches_oracle_observables():
    spec = bloch_cell(I.PREC_C128)
    inp = bloch_inputs(spec)
    sysm = _system(spec, inp)
    got = sysm.observe(1.0, 1.25)
    sysm.close()
    ref = oracle.System(spec, inp).observables(inp.psi0, 1.0, 1.25)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_unstable_substep_is_refused():
    from paper_1912_07921_gb300._lib import TdksError
    spec = I.medium_molecule(prec=I.PREC_C64, nx=24, ny=24, nz=24, n_orb=8)
    inp = I.make_inputs(spec)
    sysm = _system(spec, inp)
    with pytest.raises(TdksError) as e:
        sysm.propagate(0.0, spec.dt, 1, 1)
    assert e.value.code == 3
    sysm.close()


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_periodic_cell_full_grid_one_step(prec):
    """Periodic cell at full size (64^3, side 10.2, 8 diamond atoms with projectors,
    velocity gauge A0 = 0.2, 6 sub-steps of the configured dt = 0.04) with 2 of its 32
    k-points x 16 bands; every value compared, current and energy records too."""
    spec = I.periodic_cell(n_k=2, prec=prec)
    inp = I.make_inputs(spec)
    t0 = 30.0
    sysm = _system(spec, inp)
    sysm.propagate(t0, spec.dt, 1, spec.substeps)
    rec = sysm.reductions(0, 1)
    psi = sysm.get_orbitals()
    sysm.close()
    o = oracle.System(spec, inp)
    psi_o, rec_o = o.propagate(inp.psi0, t0, spec.dt, 1, spec.substeps)
    if prec == I.PREC_C128:
        assert rel_err(psi, psi_o) < 1e-12
        np.testing.assert_allclose(rec, rec_o, rtol=1e-12, atol=1e-12 * np.abs(rec_o).max())
    else:
        assert rel_err(psi, psi_o) < 1e-5
        # <phi|H|phi> from an FP32 H phi: the kinetic terms (up to K_max ~ 315 Ha here) cancel
        # down to ~0.45 Ha per orbital, so the relative error is ~eps32 * K_max / e ~ 4e-5
        assert abs(rec[0, 2] - rec_o[0, 2]) < 2e-4 * abs(rec_o[0, 2])
        assert np.max(np.abs(rec[0, 4:7] - rec_o[0, 4:7])) < 1e-4 * np.max(np.abs(rec_o[0, 4:7]))


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_periodic_current_includes_the_projectors_commutator(prec):
    """The periodic cell's recorded current is the full -(1/Omega) <i[H, r]> (Sec.
    "Conductivities", eqn. current_density): the local part and the projectors' commutator,
    against the oracle's velocity expectation; without the commutator it would differ."""
    spec = bloch_cell(prec, n_orb=5 if prec == I.PREC_C64 else 3)
    inp = bloch_inputs(spec)
    psi = inp.psi0
    if prec == I.PREC_C64:
        inp.psi0 = psi.astype(np.complex64).astype(np.complex128)
    sysm = _system(spec, inp)
    got = sysm.observe(0.0, 0.45)
    sysm.close()
    o = oracle.System(spec, inp)
    _, A = o.field(0.45)
    omega = spec.nx * spec.ny * spec.nz * spec.h ** 3
    full = -o.velocity(A, inp.psi0) / omega
    local = -o.velocity(A, inp.psi0, with_nonlocal=False) / omega
    scale = np.abs(full).max()
    assert np.abs(full - local).max() > 1e-3 * scale
    tol = 1e-12 if prec == I.PREC_C128 else 1e-4
    assert np.abs(got[4:7] - full).max() < tol * scale


@pytest.mark.parametrize("prec,order", [(I.PREC_C128, 4), (I.PREC_C128, 8), (I.PREC_C64, 4)])
def test_heat_current_matches_oracle(prec, order):
    """The kinetic heat current of Sec. "Conductivities" (eqn. KEcurrent; the reading with the
    last pair antisymmetric, covariant derivatives) of a periodic cell in the velocity gauge: the
    GPU's cell integral (composed second differences, no mixed derivatives) against the oracle's
    pointwise formula."""
    spec = bloch_cell(prec, fd_order=order, n_k=2)
    inp = bloch_inputs(spec)
    psi = I.random_orbitals(spec, 17) * 0.2 + inp.psi0
    if prec == I.PREC_C64:
        psi = psi.astype(np.complex64).astype(np.complex128)
    inp.psi0 = psi
    sysm = _system(spec, inp)
    got = sysm.heat_current(0.6)
    sysm.close()
    o = oracle.System(spec, inp)
    _, A = o.field(0.6)
    assert np.abs(A).max() > 0
    ref = o.heat_current(A, psi)
    tol = 1e-11 if prec == I.PREC_C128 else 1e-6
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (got, ref)


def test_heat_current_refuses_finite_boxes():
    from paper_1912_07921_gb300._lib import TdksError
    spec = ragged_molecule(I.PREC_C128)
    sysm = _system(spec, I.make_inputs(spec))
    with pytest.raises(TdksError) as e:
        sysm.heat_current(0.0)
    assert e.value.code == 1
    sysm.close()
