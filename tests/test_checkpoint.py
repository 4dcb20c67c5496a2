"""Checkpoint round trip and basis check, on CPU with a stand-in context (no GPU needed)."""
import numpy as np
import pytest

from paper_1211_1446_gb300 import checkpoint


class _Ctx:
    """The attributes of a Context that checkpoints read: nk, ncomp, grid, basis(ik)."""

    def __init__(self, nk, ncomp, grid, millers):
        self.nk, self.ncomp, self.grid, self._m = nk, ncomp, grid, millers

    def basis(self, ik):
        return self._m[ik]


def test_checkpoint_round_trip_and_basis_check(tmp_path):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    millers = [rng.integers(-3, 4, (5, 3)).astype(np.int32), rng.integers(-3, 4, (7, 3)).astype(np.int32)]
    ctx = _Ctx(2, 4, (12, 12, 12), millers)
    xs = [torch.from_numpy(rng.standard_normal((3, 4, n)) + 1j * rng.standard_normal((3, 4, n))) for n in (5, 7)]
    lams = [np.array([-1.0, -0.5, 0.25]), np.array([-2.0, 0.0, 1.0])]
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, ctx, xs, lams, scf_iteration=7, residual=1.5e-5)
    ys, ls, meta = checkpoint.load(path, ctx, device="cpu")
    for a, b in zip(xs, ys):
        assert b.dtype == torch.complex128 and torch.equal(a, b)
    for a, b in zip(lams, ls):
        assert np.array_equal(a, b)
    assert int(meta["scf_iteration"]) == 7 and float(meta["residual"]) == 1.5e-5
    other = _Ctx(2, 4, (12, 12, 12), [millers[0], millers[1][::-1]])
    with pytest.raises(ValueError, match="k-point 1"):
        checkpoint.load(path, other, device="cpu")
    with pytest.raises(ValueError, match="another context"):
        checkpoint.load(path, _Ctx(2, 2, (12, 12, 12), millers), device="cpu")
    with pytest.raises(ValueError):
        checkpoint.save(path, ctx, xs[:1], lams)
