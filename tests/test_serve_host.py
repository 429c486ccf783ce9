"""Host logic of the serving loop (binding.serve) against a fake context: no
GPU.  Every queued slice is read out exactly once into its own output, the
compaction at the end of the queue only moves running slices onto free
slots and never leaves a running slice outside the launched range, and the
launched-slot count is reset when the loop ends."""
import random

from paper_1411_5057_gb300 import binding as Bd


class FakeCtx:
    """Slots hold (slice index, outer steps still needed, outer steps done);
    every run advances the running slices in the launched slots by one outer
    step per `steps_per_outer` macro steps."""

    def __init__(self, batch, need, steps_per_outer=8):
        self.batch, self.need, self.spo = batch, need, steps_per_outer
        self.slots = [None] * batch
        self.active = 0
        self.moves = 0

    def set_active_slots(self, k):
        assert 0 <= k <= self.batch
        self.active = 0 if k == self.batch else k

    def slot_load(self, s, mask, b, lam, lam_tv, x0=None, eps=0.0):
        assert self.slots[s] is None or self.slots[s][3], "loading over a running slice"
        self.slots[s] = [b, self.need[b], 0, False]

    def slot_retire(self, s):
        if self.slots[s] is not None:
            self.slots[s][3] = True

    def slot_move(self, src, dst):
        assert src != dst and self.slots[src] is not None and not self.slots[src][3]
        assert self.slots[dst] is None or self.slots[dst][3], "moving onto a running slice"
        self.slots[dst] = list(self.slots[src])
        self.slots[src][3] = True
        self.moves += 1

    def run_steps(self, params, macro_steps):
        k = self.active or self.batch
        for s, v in enumerate(self.slots):
            running = v is not None and not v[3]
            if s >= k:
                assert not running, f"slot {s} runs outside the launched {k}"
                continue
            if running:
                v[2] += macro_steps // self.spo
                if v[2] >= v[1]:
                    v[2] = v[1]
                    v[3] = True

    def slot_status(self, with_pcg=False):
        done = [1 if (v is None or v[3]) else 0 for v in self.slots]
        od = [0 if v is None else v[2] for v in self.slots]
        rel = [0.0] * self.batch
        pc = [10 * x for x in od]
        return (done, od, rel, pc) if with_pcg else (done, od, rel)

    def slot_get(self, s, out):
        out.append(self.slots[s][0])


def _serve(compact, seed=0, q=23, batch=8):
    rnd = random.Random(seed)
    need = [rnd.randint(2, 40) for _ in range(q)]
    ctx = FakeCtx(batch, need)
    outs = [[] for _ in range(q)]
    cnt, pcg = {}, [0] * q
    steps = Bd.serve(ctx, [None] * q, list(range(q)), [0.0] * q, [0.0] * q, Bd.Params(), outs, chunk=16,
                     max_outer=10 ** 6, counters=cnt, pcg_steps=pcg, compact=compact)
    return ctx, need, outs, steps, pcg, cnt


def test_every_slice_read_out_once_with_compaction():
    for seed in range(5):
        ctx, need, outs, steps, pcg, cnt = _serve(True, seed)
        assert [o for o in outs] == [[i] for i in range(len(need))]
        assert steps == need and pcg == [10 * x for x in need]
        assert cnt["moves"] == ctx.moves and cnt["loads"] == len(need)
        assert ctx.active == 0


def test_compaction_changes_no_outcome():
    a = _serve(False, 3)
    b = _serve(True, 3)
    assert a[2] == b[2] and a[3] == b[3] and a[4] == b[4]
    assert a[5]["moves"] == 0 and b[5]["moves"] > 0


def test_bucket_sequence():
    for batch in (1, 2, 7, 16, 304):
        prev = batch
        for act in range(batch, 0, -1):
            k = Bd._bucket(batch, act)
            assert act <= k <= prev
            prev = k
        assert Bd._bucket(batch, 1) == 1
