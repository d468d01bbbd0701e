"""The access patterns of in-place streaming (goc_exec.streaming = 1), checked
on the host: in every step each slot of the single population buffer is read
and then written by one and the same node, so one launch may overwrite its
own input, and the two layouts carry every post-collision population to the
node that pulls it.  The rules below restate the layouts of the library's
in-place step (link velocities of the D2Q9 lattice, Eq. 1a/1b):

  layout C  slot (x, a) holds the population of node x along link a (f^0);
  layout S  the post-collision population of node x along link a is at
            (x, opp(a));
  layout T  it is at (x + e_a, a), or at (x, opp(a)) when x + e_a is outside.

A step reading C or T writes S; a step reading S writes T.  The D2Q5
populations of the MIE (Appendix G) follow the same rules with their five
links."""
import itertools

import pytest

D2Q9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
D2Q5 = D2Q9[:5]
E, OPP = D2Q9, None   # the link set under test (set by each test)


def use(links):
    global E, OPP
    E = links
    OPP = [E.index((-ex, -ey)) for ex, ey in E]


def inside(x, y, nx, ny, px, py):
    """The node (x, y), wrapped on periodic axes, or None outside a wall."""
    if not 0 <= x < nx:
        if not px:
            return None
        x %= nx
    if not 0 <= y < ny:
        if not py:
            return None
        y %= ny
    return x, y


def slot_of(layout, node, a, dims):
    """Where the post-collision population of node along link a is kept."""
    x, y = node
    if layout == "C":
        return (x, y, a)
    if layout == "S":
        return (x, y, OPP[a])
    d = inside(x + E[a][0], y + E[a][1], *dims)
    return (d[0], d[1], a) if d else (x, y, OPP[a])


def pulled(node, a, dims):
    """The population the pull step hands node along link a: from the
    upstream node, or the node's own reversed one at a wall (bounce-back)."""
    x, y = node
    src = inside(x - E[a][0], y - E[a][1], *dims)
    return (src, a) if src else (node, OPP[a])


def reads(layout, node, dims, first_step):
    if first_step:                        # f^0 is read in place
        return {slot_of("C", node, a, dims) for a in range(len(E))}
    return {slot_of(layout, *pulled(node, a, dims), dims) for a in range(len(E))}


def writes(layout_in, node, dims):
    out = "T" if layout_in == "S" else "S"
    return {slot_of(out, node, a, dims) for a in range(len(E))}


CASES = [(5, 4, False, False), (5, 4, True, False), (5, 4, False, True), (6, 3, True, True),
         (1, 4, True, False), (3, 1, False, True), (2, 2, True, True), (7, 6, False, False)]


@pytest.mark.parametrize("links", [D2Q9, D2Q5], ids=["d2q9", "d2q5"])
@pytest.mark.parametrize("nx, ny, px, py", CASES)
@pytest.mark.parametrize("layout, first", [("C", True), ("S", False), ("T", False)])
def test_each_slot_is_read_and_written_by_one_node(nx, ny, px, py, layout, first, links):
    use(links)
    dims = (nx, ny, px, py)
    nodes = list(itertools.product(range(nx), range(ny)))
    owner_r, owner_w = {}, {}
    for n in nodes:
        r, w = reads(layout, n, dims, first), writes(layout, n, dims)
        assert len(r) == len(E) and len(w) == len(E)   # one distinct slot per link each
        for s in r:
            assert owner_r.setdefault(s, n) == n     # no slot is read by two nodes
        for s in w:
            assert owner_w.setdefault(s, n) == n     # no slot is written by two nodes
        assert r == w                                # a node writes exactly the slots it read
    every = {(x, y, a) for x, y in nodes for a in range(len(E))}
    assert set(owner_w) == every                     # the layouts fill the buffer


@pytest.mark.parametrize("links", [D2Q9, D2Q5], ids=["d2q9", "d2q5"])
@pytest.mark.parametrize("nx, ny, px, py", CASES)
def test_alternating_layouts_deliver_every_population_to_its_puller(nx, ny, px, py, links):
    """Three steps on symbolic populations: the value each node pulls is the
    post-collision population the two-buffer pull step would hand it."""
    use(links)
    dims = (nx, ny, px, py)
    nodes = list(itertools.product(range(nx), range(ny)))
    buf = {(x, y, a): ("f0", (x, y), a) for x, y in nodes for a in range(len(E))}
    layout, first = "C", True
    for step in range(1, 4):
        new = {}
        for n in nodes:
            if first:
                got = [buf[slot_of("C", n, a, dims)] for a in range(len(E))]
                assert got == [("f0", n, a) for a in range(len(E))]
            else:
                for a in range(len(E)):
                    src, b = pulled(n, a, dims)
                    assert buf[slot_of(layout, src, b, dims)] == (step - 1, src, b)
            for a in range(len(E)):                       # post-collision population of step `step`
                new[slot_of("T" if layout == "S" else "S", n, a, dims)] = (step, n, a)
        buf.update(new)
        layout, first = ("T" if layout == "S" else "S"), False
