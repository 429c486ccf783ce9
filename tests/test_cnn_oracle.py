"""Pins for the FP64 CNN oracle: brute-force convolution, adjointness, and
gradients against central differences of the loss."""
import numpy as np

import firls_synth as fs
from oracle import cnn_oracle as C


def test_conv_matches_bruteforce():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 5, 6, 3))
    w = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    z = C.conv3x3(a, w, b)
    for bb in range(2):
        for y in range(5):
            for x in range(6):
                for o in range(4):
                    s = b[o]
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            if 0 <= y + dy < 5 and 0 <= x + dx < 6:
                                s += np.dot(a[bb, y + dy, x + dx], w[dy + 1, dx + 1, :, o])
                    assert abs(z[bb, y, x, o] - s) < 1e-12


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((1, 7, 5, 3))
    w = rng.standard_normal((3, 3, 3, 2))
    dz = rng.standard_normal((1, 7, 5, 2))
    da, dw, db = C.conv3x3_backward(a, w, dz)
    # <conv(a), dz> is linear in a: its gradient is da
    lhs = np.sum(C.conv3x3(a, w, np.zeros(2)) * dz)
    assert abs(lhs - np.sum(a * da)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * dw)) < 1e-10 * abs(lhs)
    assert np.allclose(db, dz.sum(axis=(0, 1, 2)))


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    n = 6
    params = [(rng.standard_normal(w.shape) * 0.3, rng.standard_normal(b.shape) * 0.1)
              for w, b in fs.cnn_init_weights(3)]
    # shrink the hidden width so the check stays fast
    small = []
    chans = [3, 4, 4, 4, 4, 4, 2]
    for l in range(6):
        small.append((params[l][0][:, :, :chans[l], :chans[l + 1]].copy(), params[l][1][:chans[l + 1]].copy()))
    atb = rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))
    mask = (rng.random((n, n)) < 0.3)
    inp = fs.cnn_input(atb[0], mask)[None]
    target = rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))
    loss, grads, _ = C.loss_and_grads(small, inp, atb, target)
    h = 1e-6
    for l in (0, 3, 5):
        w, b = small[l]
        for idx in [(0, 1, 0, 1), (1, 1, 2, 0), (2, 0, 1, 1)]:
            wp = [(x[0].copy(), x[1].copy()) for x in small]
            wm = [(x[0].copy(), x[1].copy()) for x in small]
            wp[l][0][idx] += h
            wm[l][0][idx] -= h
            fd = (C.loss_and_grads(wp, inp, atb, target)[0] - C.loss_and_grads(wm, inp, atb, target)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) < 1e-5 * max(1.0, abs(fd)), (l, idx, fd, grads[l][0][idx])
        bp = [(x[0].copy(), x[1].copy()) for x in small]
        bm = [(x[0].copy(), x[1].copy()) for x in small]
        bp[l][1][1] += h
        bm[l][1][1] -= h
        fd = (C.loss_and_grads(bp, inp, atb, target)[0] - C.loss_and_grads(bm, inp, atb, target)[0]) / (2 * h)
        assert abs(fd - grads[l][1][1]) < 1e-5 * max(1.0, abs(fd))


def test_untrained_network_returns_zero_filled():
    n = 8
    rng = np.random.default_rng(4)
    atb = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    acts = C.forward(fs.cnn_init_weights(0), fs.cnn_input(atb, np.ones((n, n)))[None])
    assert np.all(acts[-1] == 0)


def test_adam_matches_closed_form_first_step():
    """First Adam step moves every parameter by lr * sign(g) (bias-corrected)."""
    params = [(np.ones((1,)), np.zeros((1,)))]
    grads = [(np.array([0.5]), np.array([-2.0]))]
    st = C.adam_init(params)
    out = C.adam_step(params, grads, st, lr=0.1)
    assert abs(out[0][0][0] - (1 - 0.1)) < 1e-7 and abs(out[0][1][0] - 0.1) < 1e-7
