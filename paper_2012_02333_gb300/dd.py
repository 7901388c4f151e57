"""Dynamic-definition driver (Sec. 4.3, Algorithm 1).

Each recursion labels every qubit active, merged or zoomed; the library
(cutqc_reconstruct_dd) merges the subcircuit tensors over the merged qubits
with the zoomed qubits fixed, reconstructs the 2^#active bins, and returns the
heaviest bins ranked in FP64.  This module keeps the list of bins of all
recursions (Algorithm 1's probability_bins, as each recursion's top-32 list)
and picks the next bin to zoom into.

Readings of the paper used here (it leaves them open):
  * recursion 1 makes the n_active lowest-numbered qubits active;
  * a zoom keeps earlier zoomed qubits, fixes the parent's active qubits at
    the chosen bin's bits, and activates the next min(n_active, #merged)
    lowest-numbered merged qubits;
  * "bfs" zooms into the heaviest bin over all recursions that has not been
    zoomed yet and still has merged qubits (a blurred landscape that sharpens
    where the probability is); "dfs" zooms into the heaviest bin of the latest
    recursion (locating solution states); ties go to the earlier recursion,
    then the lower bin index.
The state (roles, top lists, zoom choices) serialises to JSON so a run can be
checkpointed and resumed.
"""
from __future__ import annotations

import json
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import torch

from . import circuits
from . import cutqc

ACTIVE, MERGED, ZOOM0, ZOOM1 = 0, 1, 2, 3


def initial_roles(n_qubits: int, n_active: int) -> List[int]:
    return [ACTIVE if q < n_active else MERGED for q in range(n_qubits)]


def zoom_roles(parent: Sequence[int], bin_index: int, n_active: int) -> List[int]:
    roles = list(parent)
    act = [q for q, r in enumerate(roles) if r == ACTIVE]
    for i, q in enumerate(act):
        roles[q] = ZOOM1 if (bin_index >> (len(act) - 1 - i)) & 1 else ZOOM0
    promote = [q for q, r in enumerate(roles) if r == MERGED][:n_active]
    for q in promote:
        roles[q] = ACTIVE
    return roles


@dataclass
class Recursion:
    roles: List[int]
    top: List[Tuple[int, float]]          # (bin index, FP64 value), heaviest first
    parent: Optional[Tuple[int, int]]     # (recursion, bin) zoomed into, None for the first
    bins: Optional[torch.Tensor] = None   # the 2^#active bins (device), if kept


@dataclass
class DDState:
    n_active: int
    strategy: str
    recursions: List[Recursion] = field(default_factory=list)
    expanded: List[Tuple[int, int]] = field(default_factory=list)

    def to_json(self) -> str:
        return json.dumps({"n_active": self.n_active, "strategy": self.strategy,
                           "expanded": self.expanded,
                           "recursions": [{"roles": r.roles, "top": r.top, "parent": r.parent}
                                          for r in self.recursions]})

    @classmethod
    def from_json(cls, text: str) -> "DDState":
        d = json.loads(text)
        st = cls(d["n_active"], d["strategy"])
        st.expanded = [tuple(x) for x in d["expanded"]]
        st.recursions = [Recursion(r["roles"], [tuple(t) for t in r["top"]],
                                   tuple(r["parent"]) if r["parent"] is not None else None)
                         for r in d["recursions"]]
        return st

    def next_zoom(self) -> Optional[Tuple[int, int]]:
        cands = range(len(self.recursions)) if self.strategy == "bfs" else [len(self.recursions) - 1]
        best = None
        done = set(map(tuple, self.expanded))
        for ri in cands:
            rec = self.recursions[ri]
            if MERGED not in rec.roles:
                continue
            for bi, v in rec.top:
                if bi < 0 or (ri, bi) in done:
                    continue
                if best is None or v > best[0]:
                    best = (v, ri, bi)
        return None if best is None else (best[1], best[2])


def run(cc: circuits.CutCircuit, tensors: Sequence[torch.Tensor], n_active: int, recursions: int,
        strategy: str = "bfs", algo: str = "auto", topk: int = 32, keep_bins: bool = True,
        state: Optional[DDState] = None, stream=None) -> DDState:
    """Run (or resume) Algorithm 1 for `recursions` recursions in total."""
    if strategy not in ("bfs", "dfs"):
        raise ValueError("strategy must be bfs or dfs")
    problem = cutqc.Problem.from_cut(cc, tensors)
    st = state or DDState(n_active, strategy)
    while len(st.recursions) < recursions:
        if not st.recursions:
            roles, parent = initial_roles(cc.n, n_active), None
        else:
            z = st.next_zoom()
            if z is None:
                break
            ri, bi = z
            st.expanded.append((ri, bi))
            roles, parent = zoom_roles(st.recursions[ri].roles, bi, n_active), (ri, bi)
        na = sum(1 for r in roles if r == ACTIVE)
        bins = torch.empty(2 ** na, dtype=problem.dtype, device=tensors[0].device)
        idx, val = cutqc.cutqc_reconstruct_dd(problem, roles, bins, topk, algo, stream)
        st.recursions.append(Recursion(roles, list(zip(idx, val)), parent, bins if keep_bins else None))
    return st
