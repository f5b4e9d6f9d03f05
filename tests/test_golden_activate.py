"""Algorithms 1 and 2 on instances worked by hand (tests/golden/activate_worked_example.txt,
and activate_cp_worked_example.txt with communication prediction): the scheduling oracle
and the library's placement code (the code the persistent kernel runs, called on the host)
must both reproduce the hand-derived placements."""
import os

import pytest

from oracle import sched

HERE = os.path.dirname(os.path.abspath(__file__))
LR = [dict(tid=0, p=30, prio=10, aff=1, score=8), dict(tid=1, p=20, prio=30, aff=-1, score=0),
      dict(tid=2, p=10, prio=20, aff=-1, score=0)]
LOAD = [0, 0]


def _cases():
    out = []
    for line in open(os.path.join(HERE, "golden", "activate_worked_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, rest = line.split(":")
        pairs, halvings = rest.split(";")
        policy, alpha = head.split()
        v = [int(x) for x in pairs.split()]
        out.append((policy, float(alpha), list(zip(v[0::2], v[1::2])), int(halvings)))
    return out


CASES = _cases()


def test_fixture_has_every_policy():
    assert [(c[0], c[1]) for c in CASES] == [("heft", 0.0), ("dada", 0.0), ("dada", 0.5), ("dada", 1.0)]


@pytest.mark.parametrize("policy,alpha,pairs,halvings", CASES)
def test_oracle_reproduces_hand_worked_activate(policy, alpha, pairs, halvings):
    if policy == "heft":
        assert sched.heft(LR, LOAD) == pairs
    else:
        assert sched.dada(LR, LOAD, alpha) == (pairs, halvings)


@pytest.mark.parametrize("policy,alpha,pairs,halvings", CASES)
def test_library_reproduces_hand_worked_activate(policy, alpha, pairs, halvings):
    import paper_1402_6601_gb300 as chol
    assert chol.sched_activate(policy, LR, LOAD, alpha=alpha) == (pairs, halvings)


LR_CP = [dict(tid=0, p=10, prio=2, aff=-1, score=0, own=[1, 1, -1], nin=2, comm=15),
         dict(tid=1, p=10, prio=1, aff=-1, score=0, own=[0, -1, -1], nin=1, comm=15)]


def _cp_cases():
    out = []
    for line in open(os.path.join(HERE, "golden", "activate_cp_worked_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, rest = line.split(":")
        pairs, halvings = rest.split(";")
        policy, alpha, cp = head.split()
        v = [int(x) for x in pairs.split()]
        out.append((policy, float(alpha), bool(int(cp)), list(zip(v[0::2], v[1::2])), int(halvings)))
    return out


@pytest.mark.parametrize("policy,alpha,cp,pairs,halvings", _cp_cases())
def test_cp_hand_worked_activate(policy, alpha, cp, pairs, halvings):
    import paper_1402_6601_gb300 as chol
    if policy == "heft":
        ref = (sched.heft_cp(LR_CP, LOAD) if cp else sched.heft(LR_CP, LOAD), 0)
    else:
        ref = sched.dada_cp(LR_CP, LOAD, alpha)
    assert ref == (pairs, halvings)
    assert chol.sched_activate(policy, LR_CP, LOAD, alpha=alpha, use_cp=cp) == (pairs, halvings)
