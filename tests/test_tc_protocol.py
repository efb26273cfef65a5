"""CPU model of the score kernel's barrier protocol (csrc/tc_topk.cu): the
producer (work items, user tiles, item-tile ring), the bound-column copier,
two MMA issuers and the select warps, each a coroutine over mbarrier-like
counters, run under random interleavings with copies landing in any order.

An mbarrier wait in the kernel is a parity wait: it asks whether the phase
with the parity of phase k has completed, so it answers correctly only
while the barrier is between phase k - 1 and phase k + 1.  The model flags
every wait that would be answered wrongly (a success with phase k still
open, or a wait on phase k once phase k + 1 has completed) and any
deadlock.  It pins two rules of the kernel:
  * the issuers split the item tiles by parity only when the S ring stages
    split with them (S a multiple of 2 bs, bs loads per item tile), so each
    stage's barriers are waited on by one issuer, phase by phase;
  * the select releases a bound-column slot only after waiting for its
    copy, so the copier, which runs on its own thread, never sees a slot
    released ahead of its copy.
With either rule dropped the model finds a wrong answer in a few hundred
schedules (the rule is not vacuous)."""
import os
import random

import pytest

KWQ, KAUX = 4, 4
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1706_01449_gb300", "csrc",
                   "tc_topk.cu")


class Hazard(Exception):
    pass


class Bar:
    def __init__(self, count, name):
        self.count, self.name, self.pending, self.done = count, name, 0, 0

    def arrive(self):
        self.pending += 1
        if self.pending == self.count:
            self.pending = 0
            self.done += 1

    def wait(self, k):
        """Parity wait for phase k (0-based): true iff the completed-phase
        count has the other parity; a hazard if that answer is wrong."""
        ok = (self.done & 1) != (k & 1)
        if ok and self.done != k + 1:
            raise Hazard(f"{self.name}: wait for phase {k} passed with {self.done} phases done")
        if not ok and self.done >= k + 2:
            raise Hazard(f"{self.name}: wait for phase {k} blocked with {self.done} phases done")
        return ok


def simulate(seed, S, bs, works, split_rule=True, select_waits_copy=True, slow=None):
    rnd = random.Random(seed)
    B = {}

    def mk(name, count):
        B[name] = Bar(count, name)

    for s in range(S):
        mk(f"b_full{s}", 1)
        mk(f"b_empty{s}", 1)
    for a in range(2):
        mk(f"a_full{a}", 1)
        mk(f"a_empty{a}", 2)  # one commit per issuer
        mk(f"acc_full{a}", 1)
        mk(f"acc_empty{a}", 1)  # the select warps, as one actor
    for a in range(KAUX):
        mk(f"aux_full{a}", 1)
        mk(f"aux_empty{a}", 1)
    for w in range(KWQ):
        mk(f"wq_full{w}", 1)
        mk(f"wq_empty{w}", 4)  # two issuers, the copier, the select
    landing = []  # copies in flight (land in any order)
    pipe = []     # tensor pipe: MMAs and commits in issue order
    split = (S % (2 * bs) == 0) if split_rule else True

    def take_work(lt):
        slot = lt % KWQ
        while not B[f"wq_full{slot}"].wait(lt // KWQ):
            yield
        B[f"wq_empty{slot}"].arrive()

    def producer():
        g = na = 0
        for lt, ntiles in enumerate(works + [None]):
            slot = lt % KWQ
            if lt >= KWQ:
                while not B[f"wq_empty{slot}"].wait(lt // KWQ - 1):
                    yield
            B[f"wq_full{slot}"].arrive()
            if ntiles is None:
                return
            asl = na & 1
            if na >= 2:
                while not B[f"a_empty{asl}"].wait((na >> 1) - 1):
                    yield
            landing.append(f"a_full{asl}")
            na += 1
            for _ in range(ntiles):
                for _h in range(bs):
                    st = g % S
                    if g >= S:
                        while not B[f"b_empty{st}"].wait(g // S - 1):
                            yield
                    landing.append(f"b_full{st}")
                    g += 1
                yield

    def copier():
        at = 0
        for lt in range(len(works) + 1):
            yield from take_work(lt)
            if lt == len(works):
                return
            for _ in range(works[lt]):
                a = at % KAUX
                if at >= KAUX:
                    while not B[f"aux_empty{a}"].wait(at // KAUX - 1):
                        yield
                    while not B[f"aux_full{a}"].wait(at // KAUX - 1):
                        yield
                landing.append(f"aux_full{a}")
                at += 1
                yield

    def issuer(mine):
        g = ld = 0
        for lt in range(len(works) + 1):
            yield from take_work(lt)
            if lt == len(works):
                return
            asl = lt & 1
            while not B[f"a_full{asl}"].wait(lt >> 1):
                yield
            for _ in range(works[lt]):
                b = g & 1
                if not ((b == mine) if split else (mine == 0)):
                    ld += bs
                    g += 1
                    continue
                for h in range(bs):
                    st = ld % S
                    while not B[f"b_full{st}"].wait(ld // S):
                        yield
                    if h == 0 and g >= 2:
                        while not B[f"acc_empty{b}"].wait((g >> 1) - 1):
                            yield
                    pipe.append(("mma", None))
                    pipe.append(("commit", f"b_empty{st}"))
                    ld += 1
                    yield
                pipe.append(("commit", f"acc_full{b}"))
                g += 1
            pipe.append(("commit", f"a_empty{asl}"))

    def select():
        g = 0
        for lt in range(len(works) + 1):
            yield from take_work(lt)
            if lt == len(works):
                return
            for _ in range(works[lt]):
                b, a = g & 1, g % KAUX
                if select_waits_copy or rnd.random() < 0.3:  # (else: only when a hit needs the columns)
                    while not B[f"aux_full{a}"].wait(g // KAUX):
                        yield
                while not B[f"acc_full{b}"].wait(g >> 1):
                    yield
                yield
                B[f"acc_empty{b}"].arrive()
                B[f"aux_empty{a}"].arrive()
                g += 1

    actors = {"producer": producer(), "copier": copier(), "issuer0": issuer(0), "issuer1": issuer(1),
              "select": select()}
    steps = 0
    while actors or landing or pipe:
        cands = list(actors) + (["land"] if landing else []) + (["pipe"] if pipe else [])
        # a slow actor takes a step only now and then (slow = {name: weight})
        choice = rnd.choices(cands, weights=[(slow or {}).get(c, 1.0) for c in cands])[0]
        if choice == "land":
            B[landing.pop(rnd.randrange(len(landing)))].arrive()
        elif choice == "pipe":
            kind, bar = pipe.pop(0)  # a commit arrives once the MMAs ahead of it are done
            if kind == "commit":
                B[bar].arrive()
        else:
            try:
                next(actors[choice])
            except StopIteration:
                del actors[choice]
        steps += 1
        if steps > 100000:
            raise Hazard("no progress: deadlock")


def _schedules(n):
    for seed in range(n):
        r = random.Random(1000 + seed)
        yield seed, [r.randint(1, 9) for _ in range(r.randint(1, 7))]


def _hazards(S, bs, n, **kw):
    found = []
    for seed, works in _schedules(n):
        try:
            simulate(seed, S, bs, works, **kw)
        except Hazard as e:
            found.append(str(e))
    return found


@pytest.mark.parametrize("S,bs", [(2, 1), (3, 1), (4, 1), (5, 1), (6, 1), (2, 2), (3, 2), (4, 2), (6, 2)])
def test_protocol_is_safe_with_the_kernel_rules(S, bs):
    assert _hazards(S, bs, 150) == []


@pytest.mark.parametrize("S,bs", [(2, 2), (3, 1), (3, 2)])
def test_splitting_tiles_without_splitting_stages_is_caught(S, bs):
    # two issuers sharing ring stages skip phases of each other's barriers
    assert _hazards(S, bs, 300, split_rule=False)


def test_releasing_a_slot_before_its_copy_is_caught():
    # a copier that falls behind sees slots released ahead of their copies
    assert _hazards(4, 1, 200, select_waits_copy=False, slow={"copier": 0.05})
    assert _hazards(4, 1, 200, select_waits_copy=True, slow={"copier": 0.05}) == []


def test_model_matches_the_kernel_source():
    # the rules the model checks are the ones the kernel states
    src = open(SRC).read()
    assert "const bool split = p.stages % (2 * bs) == 0;" in src
    assert "mbar_init(&ctl->a_empty[a], 2);" in src
    assert "mbar_init(&ctl->wq_empty[w], 3 + kEpiWarps);" in src
    i = src.index("ok = __all_sync(kFull, mbar_wait(&ctl->aux_full[as], aph, gd));")
    j = src.index("ok = __all_sync(kFull, mbar_wait(&ctl->acc_full[b], (uint32_t)((g >> 1) & 1), gd));")
    assert i < j  # the select waits for the copy first, on every tile
