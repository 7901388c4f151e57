"""Host logic of the dynamic-definition driver (Algorithm 1), no GPU: the role
transitions match the Figure 7 walk-through and the oracle's reading, the
BFS / DFS zoom choice and its tie rule, and checkpoint / resume through JSON."""
import pytest

from oracle import reconstruct as rc


@pytest.fixture(scope="module")
def dd():
    from paper_2012_02333_gb300 import dd
    return dd


def test_roles_follow_figure7(dd):
    # 4 qubits, 1 active: recursion 1 merges qubits 2..4 (1-based), recursion 2
    # holds qubit 1 at |1> and merges qubits 3, 4, and so on
    r = dd.initial_roles(4, 1)
    assert r == [0, 1, 1, 1]
    r = dd.zoom_roles(r, 1, 1)
    assert r == [3, 0, 1, 1]
    r = dd.zoom_roles(r, 1, 1)
    assert r == [3, 3, 0, 1]
    r = dd.zoom_roles(r, 1, 1)
    assert r == [3, 3, 3, 0]


def test_roles_agree_with_the_oracle_reading(dd):
    import random
    rng = random.Random(3)
    for _ in range(50):
        n = rng.randint(3, 12)
        na = rng.randint(1, n)
        a, b = dd.initial_roles(n, na), rc.initial_roles(n, na)
        assert a == b
        for _ in range(4):
            k = sum(1 for x in a if x == 0)
            if k == 0:
                break
            idx = rng.randrange(2 ** k)
            a, b = dd.zoom_roles(a, idx, na), rc.zoom_roles(b, idx, na)
            assert a == b


def test_next_zoom_bfs_dfs_and_ties(dd):
    st = dd.DDState(1, "bfs")
    st.recursions.append(dd.Recursion([0, 1, 1], [(0, 0.6), (1, 0.4)], None))
    assert st.next_zoom() == (0, 0)
    st.expanded.append((0, 0))
    st.recursions.append(dd.Recursion([2, 0, 1], [(1, 0.35), (0, 0.25)], (0, 0)))
    # bfs: the unexpanded bin 1 of recursion 0 (0.4) beats recursion 1's best
    assert st.next_zoom() == (0, 1)
    st.strategy = "dfs"
    assert st.next_zoom() == (1, 1)
    # ties: earlier recursion first
    st2 = dd.DDState(1, "bfs")
    st2.recursions.append(dd.Recursion([0, 1], [(0, 0.5), (1, 0.5)], None))
    st2.recursions.append(dd.Recursion([2, 0], [(1, 0.5)], (0, 9)))
    assert st2.next_zoom() == (0, 0)
    # a recursion with no merged qubits left cannot be zoomed into
    st3 = dd.DDState(1, "bfs")
    st3.recursions.append(dd.Recursion([3, 0], [(0, 0.9)], None))
    assert st3.next_zoom() is None


def test_state_json_round_trip(dd):
    st = dd.DDState(2, "bfs")
    st.recursions.append(dd.Recursion([0, 0, 1, 1], [(3, 0.5), (1, 0.25)], None))
    st.recursions.append(dd.Recursion([3, 3, 0, 0], [(2, 0.3)], (0, 3)))
    st.expanded.append((0, 3))
    back = dd.DDState.from_json(st.to_json())
    assert back.to_json() == st.to_json()
    assert back.next_zoom() == st.next_zoom()
