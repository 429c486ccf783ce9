"""The allocation-free A^H A entry point against the context-based one.

firls_apply_AHA_noalloc exists for callers that must not allocate device
memory (a host framework's memory pool, a real-time loop, a plug-in handed
only its buffers); it keeps its scratch in fixed device arrays instead.
Called here through the C ABI, twice in a row with different inputs and then
at another size, it must reproduce firls_apply_AHA (same kernels) and the FP64
oracle's A^H A = F^H R^T R F (Sec. 5.4) within the operator tolerance used by
the other parity tests.  A last test calls it from several host threads
(whole calls serialised by the callers, as the header requires) and checks
each result.
The file name makes pytest collect it last.
"""
import ctypes
import threading

import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 2e-5


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def _rel(a, b):
    a = a.detach().cpu().numpy().astype(np.complex128)
    b = b.detach().cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inputs(n, B, seed):
    rng = np.random.default_rng(seed)
    masks = np.stack([fs.vd_mask(n, 0.25, seed + s) for s in range(B)])
    d = rng.standard_normal((B, n, n)) + 1j * rng.standard_normal((B, n, n))
    return torch.from_numpy(masks).cuda(), torch.from_numpy(d).to(torch.complex64).cuda()


def _noalloc(F, n, B, mask, d, q, stream):
    lib = F.lib()
    return lib.firls_apply_AHA_noalloc(n, B, ctypes.c_void_p(mask.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                       ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_context_entry_point(F):
    stream = torch.cuda.current_stream()
    for n, B, seed in ((256, 4, 1), (256, 4, 2), (96, 3, 3)):  # two calls in a row, then another size
        mask, d = _inputs(n, B, seed)
        ctx = F.Context(n, batch=B)
        ctx.set_operator(mask, F.PSI_TV)
        q_ref = torch.empty_like(d)
        ctx.apply_AHA(d, q_ref)
        q = torch.full_like(d, float("nan"))
        assert _noalloc(F, n, B, mask, d, q, stream) == 0
        torch.cuda.synchronize()
        assert _rel(q, q_ref) < TOL_OP, (n, seed)
        mh, dh = mask.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.complex128)
        qh = q.cpu().numpy().astype(np.complex128)
        for s in range(B):
            ref = O.op_AH(O.op_A(dh[s], mh[s]), mh[s], False)
            assert np.linalg.norm(qh[s] - ref) / np.linalg.norm(ref) < TOL_OP, (n, seed, s)
        ctx.close()


def test_noalloc_rejects_oversize_and_bad_args(F):
    stream = torch.cuda.current_stream()
    mask, d = _inputs(64, 1, 5)
    q = torch.empty_like(d)
    lib = F.lib()
    big = 1 + (1 << 20) // (512 * 512)  # batch * n^2 above FIRLS_NOALLOC_MAX_ELEMS
    assert _noalloc(F, 512, big, mask, d, q, stream) == 2
    assert _noalloc(F, 100, 1, mask, d, q, stream) == 2
    assert _noalloc(F, 64, 65, mask, d, q, stream) == 2
    assert lib.firls_apply_AHA_noalloc(64, 1, None, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream)) == 1


def test_noalloc_calls_from_several_host_threads(F):
    """Four host threads, each on its own stream, start together on a size not
    used before.  The scratch arrays are shared, so, as the header requires,
    the callers serialise whole calls (a lock around call and stream
    synchronisation); whichever thread comes first makes the size's set-up."""
    n, B = 128, 2
    inputs = [_inputs(n, B, 20 + i) for i in range(4)]
    outs = [torch.full_like(d, float("nan")) for _, d in inputs]
    streams = [torch.cuda.Stream() for _ in inputs]
    torch.cuda.synchronize()
    lock = threading.Lock()
    codes = [None] * 4
    start = threading.Barrier(4)

    def work(i):
        mask, d = inputs[i]
        start.wait()
        with lock:
            codes[i] = _noalloc(F, n, B, mask, d, outs[i], streams[i])
            streams[i].synchronize()

    threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert codes == [0, 0, 0, 0]
    for (mask, d), q in zip(inputs, outs):
        mh, dh = mask.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.complex128)
        qh = q.cpu().numpy().astype(np.complex128)
        for s in range(B):
            ref = O.op_AH(O.op_A(dh[s], mh[s]), mh[s], False)
            assert np.linalg.norm(qh[s] - ref) / np.linalg.norm(ref) < TOL_OP
