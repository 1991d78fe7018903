"""Host-side logic that needs no GPU: the real-field projection of the optimal-perturbation
iteration (adjoint.optimal_perturbation)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_2481_gb300 import adjoint as A  # noqa: E402


def test_real_field_projection_of_the_m0_line():
    """The m = 0 line of a real vector field satisfies d_+(0,k) = conj d_-(0,-k) and
    d_z(0,k) = conj d_z(0,-k); the projection enforces exactly that, leaves m > 0 alone, is
    idempotent, and keeps a line that already has the symmetry."""
    rng = np.random.default_rng(4)
    shape = (3, 6, 4, 9)   # [c][r][m][k], K = 4
    d = torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    p = A._real_field_m0(d)
    line = p[:, :, 0, :].numpy()
    assert np.array_equal(line[0], np.conj(line[1][:, ::-1]))
    assert np.array_equal(line[2], np.conj(line[2][:, ::-1]))
    assert np.all(line[2][:, 4].imag == 0)
    assert torch.equal(p[:, :, 1:, :], d[:, :, 1:, :])
    assert torch.equal(A._real_field_m0(p), p)
    # the projection is the orthogonal one: the removed part is orthogonal to every symmetric line
    r = (d - p)[:, :, 0, :].numpy()
    q = A._real_field_m0(torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape)))
    assert abs(np.real(np.vdot(r, q[:, :, 0, :].numpy()))) <= 1e-12 * np.linalg.norm(r) * np.linalg.norm(q.numpy())
