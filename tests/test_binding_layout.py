"""Host-side layout conversion of the Python binding on CPU: System.pack turns host orbitals
[k][z][y][x][orb] into the library's packed batches [k][batch][z][y][x][j] (orbital
o = batch * BS + j, zero-padded to whole batches, complex64 for complex64 systems) and
System.unpack inverts it.  Run on a stand-in that reports the layout as the library does."""
import numpy as np
import pytest

from paper_1912_07921_gb300.system import System


class Stand:
    def __init__(self, shape, bs, eb):
        self.shape, self._bs, self._eb = shape, bs, eb

    def layout(self):
        nb = -(-self.shape[-1] // self._bs)
        return self._bs, nb, self._eb, 0


@pytest.mark.parametrize("n_orb,bs,eb", [(5, 4, 16), (8, 4, 16), (11, 8, 8), (1, 8, 8)])
def test_pack_places_every_orbital_in_its_batch_and_pads_with_zeros(n_orb, bs, eb):
    shape = (2, 3, 4, 5, n_orb)
    rng = np.random.default_rng(n_orb)
    psi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    st = Stand(shape, bs, eb)
    packed = System.pack(st, psi)
    nb = -(-n_orb // bs)
    assert packed.shape == (2, nb, 3, 4, 5, bs)
    assert packed.dtype == (np.complex64 if eb == 8 else np.complex128)
    for o in range(nb * bs):
        got = packed[:, o // bs, ..., o % bs]
        want = psi[..., o] if o < n_orb else np.zeros(shape[:-1])
        np.testing.assert_array_equal(got, want.astype(packed.dtype))
    back = System.unpack(st, packed)
    tol = 0 if eb == 16 else 1e-6
    np.testing.assert_allclose(back, psi, rtol=0, atol=tol * np.abs(psi).max())
