"""Seeded input generators (workloads.py) used by the parity tests and the
bench: shapes and structure of the paper's random family at the widths of
its App. A validation sets."""
import pytest

from paper_2304_14969_gb300 import workloads as W


@pytest.mark.parametrize("w,d", [(6, 6), (12, 6), (18, 6), (12, 12), (18, 12), (18, 18), (15, 15), (19, 10)])
def test_paper_family_at_appendix_widths(w, d):
    """Width w on a ceil(sqrt(w))-column grid with the last row partial: one
    U3 per qubit per layer, couplers only between existing sites, nearest
    neighbours on the grid, no qubit twice in a layer's couplers."""
    rows, cols = W.grid_shape(w)
    assert rows * cols >= w > (rows - 1) * cols
    g = W.paper_random_circuit(rows, cols, d, seed=w * 10 + d, n=w)
    u3 = [x for x in g if x.name == "u3"]
    assert len(u3) == w * d
    layer_start = [i for i, x in enumerate(g) if x.name == "u3" and x.qubits[0] == 0]
    assert len(layer_start) == d
    for li, s0 in enumerate(layer_start):
        end = layer_start[li + 1] if li + 1 < d else len(g)
        cpl = [x for x in g[s0:end] if x.name != "u3"]
        used = set()
        for x in cpl:
            a, b = x.controls[0], x.qubits[0]
            assert 0 <= a < w and 0 <= b < w
            ra, ca = divmod(a, cols)
            rb, cb = divmod(b, cols)
            assert abs(ra - rb) + abs(ca - cb) == 1
            assert a not in used and b not in used
            used |= {a, b}


def test_paper_family_full_grid_unchanged():
    """n = rows * cols gives the same circuit as leaving n out."""
    a = W.paper_random_circuit(3, 4, 5, seed=11)
    b = W.paper_random_circuit(3, 4, 5, seed=11, n=12)
    assert [(x.name, x.qubits, x.params, x.controls) for x in a] == [(x.name, x.qubits, x.params, x.controls) for x in b]
