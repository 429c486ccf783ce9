"""Failure handling at the C ABI: inputs rejected before any launch, PCG
breakdowns reported per slice, and a bounded device wait that runs out.

The failures are made on the host (an empty mask, a NaN in the k-space) or by
the library's own test form of the ILU kernel, whose waits give up at once
with no copy in flight.  No GPU fault, trap or hang is involved.
"""
import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-4


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def _problems(n=64, seeds=(31, 32, 33)):
    return [fs.make_problem(n, 0.25, 0.01, s, real=False, psi=fs.PSI_TV | fs.PSI_DB4, levels=3, lam=5e-4,
                            lam_tv=1e-3) for s in seeds]


def _dev(probs):
    masks = torch.from_numpy(np.stack([p.mask for p in probs])).cuda()
    b = torch.from_numpy(np.stack([p.b for p in probs]).astype(np.complex64)).cuda()
    return masks, b


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_empty_mask_rejected(F):
    probs = _problems()
    masks, _ = _dev(probs)
    masks[1].zero_()
    ctx = F.Context(64, batch=3)
    with pytest.raises(F.FirlsError) as e:
        ctx.set_operator(masks, F.PSI_TV | F.PSI_DB4, 3)
    assert e.value.status == 1
    # the operator counts as not set: a solve is out of order
    b = torch.zeros((3, 64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FirlsError) as e:
        ctx.solve(b, F.make_params(1, 1, lam=5e-4, lam_tv=1e-3))
    assert e.value.status == 7
    ctx.close()


def test_empty_mask_rejected_by_slot_load(F):
    probs = _problems()
    masks, b = _dev(probs)
    ctx = F.Context(64, batch=2)
    ctx.set_operator(masks[:2], F.PSI_TV | F.PSI_DB4, 3)
    empty = torch.zeros_like(masks[0])
    with pytest.raises(F.FirlsError) as e:
        ctx.slot_load(0, empty, b[0], 5e-4, 1e-3)
    assert e.value.status == 1
    ctx.slot_load(1, masks[1], b[1], 5e-4, 1e-3)
    done, od, _ = ctx.slot_status()
    assert done[0] == 1 and done[1] == 0          # the rejected slot stays retired
    ctx.run(F.make_params(2, 5, lam=5e-4, lam_tv=1e-3))
    done, od, _ = ctx.slot_status()
    assert od[0] == 0 and od[1] == 2
    ctx.close()


def test_nonfinite_k_space_is_a_breakdown_of_that_slice_only(F):
    probs = _problems()
    masks, b = _dev(probs)
    i, j = np.argwhere(probs[1].mask)[3]
    b[1, i, j] = complex(float("nan"), 0.0)
    params = F.make_params(4, 10, lam=5e-4, lam_tv=1e-3)
    ctx = F.Context(64, batch=3)
    ctx.set_operator(masks, F.PSI_TV | F.PSI_DB4, 3)
    out = torch.empty_like(b)
    with pytest.raises(F.FirlsError) as e:
        ctx.solve(b, params, out=out, stats=True)
    assert e.value.status == 6
    torch.cuda.synchronize()
    # the other slices match a batch that never held the bad one, bit for bit
    keep = torch.tensor([0, 2], device="cuda")
    ref_ctx = F.Context(64, batch=2)
    ref_ctx.set_operator(masks[keep].contiguous(), F.PSI_TV | F.PSI_DB4, 3)
    ref = ref_ctx.solve(b[keep].contiguous(), params)
    assert torch.equal(out[keep], ref)
    # and the oracle
    for k, s in ((0, 0), (2, 2)):
        x_ref, _ = O.firls_problem(probs[s], outer=4, inner=10)
        assert _rel(out[k].cpu().numpy().astype(np.complex128), x_ref) < TOL_SOLVE
    # the bad slice was not iterated: it holds its start A^H b (non-finite)
    assert not torch.isfinite(torch.view_as_real(out[1])).all()
    ctx.close()
    ref_ctx.close()


def test_zero_k_space_gives_the_exact_zero(F):
    probs = _problems()
    masks, b = _dev(probs)
    b[0].zero_()
    ctx = F.Context(64, batch=3)
    ctx.set_operator(masks, F.PSI_TV | F.PSI_DB4, 3)
    out, st = ctx.solve(b, F.make_params(3, 10, lam=5e-4, lam_tv=1e-3), stats=True)
    assert st["n_breakdown"] == 0
    assert torch.count_nonzero(out[0]) == 0
    ctx.close()


def test_bounded_wait_running_out_is_reported(F):
    """The ILU kernel's test form: no copy issued, every wait gives up after
    one poll.  The solve returns FIRLS_E_DEVICE_TIMEOUT; the context then
    solves normally again."""
    probs = _problems(seeds=(41, 42))
    masks, b = _dev(probs)
    params = F.make_params(2, 5, lam=5e-4, lam_tv=1e-3)
    ctx = F.Context(64, batch=2)
    ctx.set_operator(masks, F.PSI_TV | F.PSI_DB4, 3)
    x_good = ctx.solve(b, params).clone()
    ctx.set_wait_test(True)
    with pytest.raises(F.FirlsError) as e:
        ctx.solve(b, params, stats=True)
    assert e.value.status == 8
    ctx.set_wait_test(False)
    x_again, st = ctx.solve(b, params, stats=True)
    assert st["n_breakdown"] == 0
    assert torch.equal(x_again, x_good)
    for s in range(2):
        x_ref, _ = O.firls_problem(probs[s], outer=2, inner=5)
        assert _rel(x_again[s].cpu().numpy().astype(np.complex128), x_ref) < TOL_SOLVE
    ctx.close()


def test_slot_and_dense_arguments_rejected(F):
    """Slot compaction and the dense solver reject bad arguments before any
    launch: launched-slot counts outside [0, batch], a slot moved onto
    itself or out of range, a dense matrix that is not 16-byte aligned, and
    tensors of the wrong size."""
    p = _problems(n=32, seeds=(41,))[0]
    ctx = F.Context(32, batch=3)
    ctx.set_operator(torch.from_numpy(np.stack([p.mask] * 3)).cuda(), p.psi, p.levels)
    for k in (-1, 4):
        with pytest.raises(F.FirlsError):
            ctx.set_active_slots(k)
    for a, b in ((1, 1), (0, 3), (-1, 0)):
        with pytest.raises(F.FirlsError):
            ctx.slot_move(a, b)
    ctx.set_active_slots(3)
    ctx.set_active_slots(0)
    with pytest.raises(F.FirlsError):   # two slices' worth of k-space for three slots
        ctx.solve(torch.zeros(2, 32, 32, dtype=torch.complex64, device="cuda"), F.make_params(1, 1, lam=1e-3))
    ctx.close()
    dc = F.DenseContext(8, 16, 2)
    A = torch.randn(2 * 8 * 16 + 1, device="cuda")
    with pytest.raises(F.FirlsError):
        dc.set_matrix(A[1:].view(2, 8, 16))      # 4 bytes past an aligned start
    dc.set_matrix(A[:-1].view(2, 8, 16))
    with pytest.raises(F.FirlsError):
        dc.solve(torch.zeros(2, 7, device="cuda"), F.make_params(1, 1, lam=0.1))
    dc.close()
