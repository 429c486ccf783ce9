"""GPU parity of the learned warm start's BF16 tensor-core CNN against the
FP64 CNN oracle.

The GPU rounds inputs, weights and every activation to BF16 and accumulates
in FP32; the oracle runs the same network in FP64 on the BF16-rounded inputs
and weights.  The remaining difference is the BF16 rounding of the five
hidden activations (relative 2^-9 each) and of the backward signals, so the
bounds are a few percent for outputs and gradients.
"""
import numpy as np
import pytest

import firls_synth as fs
from oracle import cnn_oracle as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FWD = 2e-2
TOL_GRAD = 5e-2


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for l, (w, b) in enumerate(fs.cnn_init_weights(seed)):
        if l == 5:  # the zero-initialised last layer would hide every earlier layer
            w = (rng.standard_normal(w.shape) * 0.05).astype(np.float32)
        out.append(((w * scale).astype(np.float32), (rng.standard_normal(b.shape) * 0.05).astype(np.float32)))
    return out


def batch_inputs(n, B, seed):
    atb, masks, tgts = [], [], []
    for s in range(B):
        p = fs.tv_db4_256(seed=seed + s, n=n)
        from oracle import firls_oracle as O
        atb.append(O.op_AH(p.b, p.mask, False))
        masks.append(p.mask)
        tgts.append(p.x0)
    return np.stack(atb), np.stack(masks), np.stack(tgts)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_inputs(atb, masks, params):
    inp = np.stack([bf16(fs.cnn_input(atb[i], masks[i])) for i in range(len(atb))])
    qp = [(bf16(w), b.astype(np.float64)) for w, b in params]  # biases stay FP32 on the GPU
    return inp, qp


@pytest.mark.parametrize("n", [64, 128], ids=["mma_sync", "tcgen05"])
def test_forward_parity(F, n):
    """n = 128 runs the convolutions on tcgen05 (TMEM accumulators), n = 64
    on mma.sync; both against the FP64 oracle."""
    B = 3
    atb, masks, _ = batch_inputs(n, B, 40)
    params = random_params(1)
    net = F.Cnn(n, B)
    net.set_params(params)
    x1 = net.forward(torch.from_numpy(atb).to(torch.complex64).cuda(), torch.from_numpy(masks).cuda())
    torch.cuda.synchronize()
    x1 = x1.cpu().numpy().astype(np.complex128)
    inp, qp = oracle_inputs(atb, masks, params)
    out = C.forward(qp, inp)[-1]
    ref = out[..., 0] + 1j * out[..., 1]
    assert rel(x1 - atb.astype(np.complex64).astype(np.complex128), ref) < TOL_FWD


@pytest.mark.parametrize("n", [64, 128], ids=["mma_sync", "tcgen05"])
def test_gradients_and_adam_step_parity(F, n):
    B = 2
    atb, masks, tgt = batch_inputs(n, B, 50)
    params = random_params(2)
    net = F.Cnn(n, B)
    net.set_params(params)
    a = torch.from_numpy(atb).to(torch.complex64).cuda()
    m = torch.from_numpy(masks).cuda()
    t = torch.from_numpy(tgt).to(torch.complex64).cuda()
    loss = net.train_step(a, m, t, lr=0.0)
    grads = net.get_grads()
    inp, qp = oracle_inputs(atb, masks, params)
    atb_q = atb.astype(np.complex64).astype(np.complex128)
    ref_loss, ref_grads, _ = C.loss_and_grads(qp, inp, atb_q, tgt.astype(np.complex64).astype(np.complex128))
    assert abs(loss - ref_loss) < TOL_FWD * ref_loss
    for l in range(6):
        assert rel(grads[l][0], ref_grads[l][0]) < TOL_GRAD, (l, rel(grads[l][0], ref_grads[l][0]))
        assert rel(grads[l][1], ref_grads[l][1]) < TOL_GRAD, (l, rel(grads[l][1], ref_grads[l][1]))
    # one Adam step with lr > 0 from the same state (the lr = 0 step above
    # advanced the step counter; reset by setting the parameters again)
    net.set_params(params)
    net.train_step(a, m, t, lr=1e-3, want_loss=False)
    after = net.get_params()
    used = net.get_grads()          # the gradients this step's update read
    for l in range(6):
        assert rel(used[l][0], ref_grads[l][0]) < TOL_GRAD, l
    # the oracle's Adam step on the same gradients, element by element: the
    # first step moves each parameter by lr g / (|g| + 1e-8) (bias-corrected
    # moments), so FP32 rounding of the update and of p leaves ~1e-8
    st = C.adam_init(qp)
    ref_after = C.adam_step([(w.astype(np.float64), b.astype(np.float64)) for w, b in params],
                            [(gw.astype(np.float64), gb.astype(np.float64)) for gw, gb in used], st, 1e-3)
    for l in range(6):
        for k in range(2):
            err = np.max(np.abs(after[l][k].astype(np.float64) - ref_after[l][k]))
            assert err < 1e-7, (l, k, err)
        assert np.max(np.abs(after[l][0] - params[l][0])) > 5e-4   # the step did move the weights


def test_training_reduces_loss(F):
    n, B = 64, 4
    atb, masks, tgt = batch_inputs(n, B, 60)
    net = F.Cnn(n, B)
    net.set_params(fs.cnn_init_weights(0))
    a = torch.from_numpy(atb).to(torch.complex64).cuda()
    m = torch.from_numpy(masks).cuda()
    t = torch.from_numpy(tgt).to(torch.complex64).cuda()
    losses = [net.train_step(a, m, t, lr=2e-3) for _ in range(60)]
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
