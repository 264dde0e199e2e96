"""Inputs f and g of a workload on a hierarchy's finest level, formed with
the quadrature rules the library exports (cc_quadrature_nodes).

f is the vector of cell averages (Eq. 4.1): exact averages on full cells,
the library's rule on cut cells.  g is the boundary-data vector of the C ABI:
exact face averages of N u on the box faces, then <<N u>> (Eq. 4.2) on each
boundary cell by the library's boundary rule.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def _bc_of(dom: W.Domain, idx: int) -> W.BC:
    return dom.box_bc[idx] if idx < 4 else dom.hole_bc[idx - 4]


def cell_averages(H, dom: W.Domain, fun, quad=None) -> np.ndarray:
    n = H.info.n
    types, _, _ = H.cell_types()
    out = np.array(W.regular_cell_averages(fun, dom, n), dtype=np.float64)
    out[types == 0] = 0.0
    q = quad if quad is not None else H.quadrature_nodes()
    vn = q["vnode"]
    vals = fun(vn[:, 0], vn[:, 1]) * vn[:, 2]
    sums = np.add.reduceat(vals, q["vptr"][:-1]) if len(vals) else np.zeros(0)
    # reduceat over empty segments is not possible here: every cut cell has nodes
    out.ravel()[q["cell"]] = sums
    return out


def boundary_data(H, dom: W.Domain, u: W.Separable, quad=None) -> np.ndarray:
    n = H.info.n
    g = [W.wall_face_data(u, dom, n)]
    q = quad if quad is not None else H.quadrature_nodes()
    bn = q["bnode"]
    tail = np.zeros(H.info.n_bd)
    if len(bn):
        vals = np.zeros(len(bn))
        for idx in np.unique(q["bbc"]):
            sel = q["bbc"] == idx
            vals[sel] = W.bc_value(u, _bc_of(dom, int(idx)), bn[sel, 0], bn[sel, 1], bn[sel, 2],
                                   bn[sel, 3])
        tail = np.add.reduceat(vals * bn[:, 4], q["bptr"][:-1])
    g.append(tail)
    return np.concatenate(g)


def problem_inputs(H, prob: W.Problem):
    """(f, g, exact cell averages of u) on the finest level of H."""
    q = H.quadrature_nodes()
    f = cell_averages(H, prob.dom, prob.f, q)
    g = boundary_data(H, prob.dom, prob.u, q)
    ue = cell_averages(H, prob.dom, prob.u, q)
    return f, g, ue
