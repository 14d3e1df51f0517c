"""Readers for the hand-worked fixtures under tests/golden/."""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class MatchCase:
    name: str
    n: int = 0
    arcs: list = field(default_factory=list)
    vlab: list = field(default_factory=list)
    k: int = 0
    parcs: list = field(default_factory=list)
    pvlab: list = field(default_factory=list)
    expect: dict = field(default_factory=dict)  # mode -> (count, rows list)

    def graph(self):
        import synth
        a = np.array(self.arcs, dtype=np.int32).reshape(-1, 3)
        return synth.Graph(self.n, a[:, 0].copy(), a[:, 1].copy(),
                           np.array(self.vlab, np.int32), a[:, 2].copy())

    def pattern(self):
        import synth
        a = np.array(self.parcs, dtype=np.int32).reshape(-1, 3)
        return synth.Pattern(self.k, a[:, 0].copy(), a[:, 1].copy(),
                             np.array(self.pvlab, np.int32), a[:, 2].copy(), self.name)


def _lines(fname):
    with open(os.path.join(GOLDEN, fname)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if line:
                yield line.split()


def match_cases(fname="matches_by_hand.txt"):
    cases, cur, mode = [], None, None
    for tok in _lines(fname):
        key = tok[0]
        if key == "case":
            cur = MatchCase(tok[1])
        elif key == "n":
            cur.n = int(tok[1])
        elif key == "arc":
            cur.arcs.append([int(x) for x in tok[1:4]])
        elif key == "vlab":
            cur.vlab = [int(x) for x in tok[1:]]
        elif key == "k":
            cur.k = int(tok[1])
        elif key == "parc":
            cur.parcs.append([int(x) for x in tok[1:4]])
        elif key == "pvlab":
            cur.pvlab = [int(x) for x in tok[1:]]
        elif key == "expect":
            mode = tok[1]
            cur.expect[mode] = (int(tok[2]), [])
        elif key == "row":
            cur.expect[mode][1].append([int(x) for x in tok[1:]])
        elif key == "end":
            cases.append(cur)
            cur = None
    return cases


def reorder_cases(fname="reorder_by_hand.txt"):
    cases, cur = [], None
    for tok in _lines(fname):
        key = tok[0]
        if key == "case":
            cur = {"name": tok[1], "arcs": []}
        elif key == "k":
            cur["k"] = int(tok[1])
        elif key == "parc":
            cur["arcs"].append((int(tok[1]), int(tok[2])))
        elif key == "order":
            cur["order"] = [int(x) for x in tok[1:]]
        elif key == "end":
            cases.append(cur)
    return cases
