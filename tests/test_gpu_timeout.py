"""The bounded pipeline waits of the TMA-fed tcgen05 near kernel (BF16
batched apply), exercised without any GPU fault: a wait limit of zero makes
every wait that is not already satisfied give up at once.  The kernel must
then drain the copies and products it had issued, free its tensor memory and
leave the outputs alone; the call returns VFD_ETIMEOUT with the caller's
output block untouched, and the next call with the default limit gives the
right products again (the error flag is reported once, the arrival counters
of the split are left consistent).
"""
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


def _tc_configs(batch, X, Y):
    """Indices of the tcgen05 candidates of the batch's near-panel tuner."""
    out = []
    n = vfd.vfd_batch_set_config(batch, 0)
    for c in range(n):
        vfd.vfd_batch_set_config(batch, c)
        try:
            vfd.vfd_batch_apply(batch, [X], [Y])
        except vfd.VfdError:
            continue
        chosen, _ = vfd.vfd_batch_tuning(batch)
        if chosen[5] == 1:
            out.append((c, chosen[2]))
    return out


def test_zero_wait_limit_times_out_and_recovers():
    m = synth.disk_mesh(14, R=1.1, jitter=0.2, seed=9)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    s, k = synth.config2_s_field(), synth.random_fourier_field(31, 0.5)
    op = vfd.vfd_assemble(mesh, s, k, 0.9, precision=vfd.VFD_BF16)
    g = torch.Generator(device="cuda").manual_seed(12)
    X = torch.randn(64, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    batch = vfd.vfd_batch_create([op])
    Yref = torch.empty_like(X)
    cands = _tc_configs(batch, X, Yref)
    assert cands, "no tcgen05 candidate ran"
    for c, split in cands:
        vfd.vfd_batch_set_config(batch, c)
        vfd.vfd_batch_set_wait_limit(batch, 1.0)
        vfd.vfd_batch_apply(batch, [X], [Yref])
        vfd.vfd_batch_set_wait_limit(batch, 0.0)
        Y = torch.full_like(X, 7.0)
        with pytest.raises(vfd.VfdError) as e:
            vfd.vfd_batch_apply(batch, [X], [Y])
        assert e.value.status == vfd.VFD_ETIMEOUT, (c, split, e.value)
        torch.cuda.synchronize()
        assert torch.all(Y == 7.0).item()          # the caller's block is untouched
        # back to the default bound: the same products as before the failure
        vfd.vfd_batch_set_wait_limit(batch, 1.0)
        Y2 = torch.empty_like(X)
        vfd.vfd_batch_apply(batch, [X], [Y2])
        torch.cuda.synchronize()
        assert torch.equal(Y2, Yref), (c, split)


def test_wait_limit_rejects_bad_values():
    m = synth.disk_mesh(6, R=1.1, jitter=0.2, seed=3)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=16)
    op = vfd.vfd_assemble(mesh, synth.config2_s_field(), synth.const_field(0.0), 0.9, precision=vfd.VFD_BF16)
    batch = vfd.vfd_batch_create([op])
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(vfd.VfdError) as e:
            vfd.vfd_batch_set_wait_limit(batch, bad)
        assert e.value.status == vfd.VFD_EINVAL
