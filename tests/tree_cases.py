"""Non-uniform plans (Sec. 3.4) built twice from the same description: as a
library tree (api.TreeNode over the package rules) and as an oracle tree
(oracle Node over the oracle rules).

A case is (names, levels) where names maps a label to how the rule is made
(a built-in, a rotation, or a variant with permuted entries), and the tree
is given as nested lists of labels.
"""
import numpy as np

from oracle import fmm as OF
from oracle import rules as OR
from paper_1507_00687_gb300 import rules as PR

P2 = np.array([[0, 1], [1, 0]])
I2 = np.eye(2)
P3 = np.array([[1, 0, 0], [0, 0, 1], [0, 1, 0]])
P3c = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]])

ORDER = {PR.ROW: "row", PR.COL: "col"}


def _oracle_base(name):
    return {"strassen": OR.strassen, "winograd": OR.winograd, "fast323": OR.fast323,
            "classical222": lambda: OR.classical(2, 2, 2), "classical121": lambda: OR.classical(1, 2, 1)}[name]()


def _package_base(name):
    return PR.get(name)


# label -> (base rule name, XU, XV, XW) or (base, "rot", times)
RECIPES = {
    "S": ("strassen", None),
    "Wg": ("winograd", None),
    "C222": ("classical222", None),
    # Strassen with the columns of B and of C permuted together (the
    # D'Alberto variant of Sec. 3.4 in its Brent-valid reading)
    "D": ("strassen", (np.eye(4), np.kron(I2, P2), np.kron(P2, I2))),
    "F": ("fast323", None),
    # the two permuted <3,2,3> variants of the non-uniform example of Sec. 3.4
    "F1": ("fast323", (np.kron(I2, P3), np.kron(P3, I2), np.kron(P3, P3))),
    "F2": ("fast323", (np.kron(I2, P3c), np.kron(P3c, I2), np.kron(P3c, P3c))),
    # rotations of <3,2,3> (App. B): <3,3,2> and <2,3,3>
    "F_r1": ("fast323", "rot1"),
    "F_r2": ("fast323", "rot2"),
}


def package_rule(label):
    base, how = RECIPES[label]
    r = _package_base(base)
    if how is None:
        return r
    if isinstance(how, str):
        for _ in range(int(how[-1])):
            r = PR.rotate(r)
        return r
    return PR.variant(r, *how, name=label)


def oracle_rule(label):
    base, how = RECIPES[label]
    r = _oracle_base(base)
    if how is None:
        return r
    if isinstance(how, str):
        for _ in range(int(how[-1])):
            r = OR.rotate(r)
        return r
    XU, XV, XW = how
    return OR.Rule(label, r.m0, r.k0, r.n0, XU @ r.U, XV @ r.V, XW @ r.W, r.order_a, r.order_b, r.order_c)


def two_level(root, children):
    """(library TreeNode, oracle Node) with `root` at level 1 and
    children[r] at level 2 under product r."""
    from paper_1507_00687_gb300 import api
    lib_rules = {lab: package_rule(lab) for lab in {root, *children}}
    orc_rules = {lab: oracle_rule(lab) for lab in {root, *children}}
    lib = api.TreeNode(lib_rules[root], [api.TreeNode(lib_rules[c], [None] * lib_rules[c].r) for c in children])
    orc = OF.Node(orc_rules[root], [OF.Node(orc_rules[c], [None] * orc_rules[c].R) for c in children])
    return lib, orc


def oracle_only_two_level(root, children):
    orc_rules = {lab: oracle_rule(lab) for lab in {root, *children}}
    return OF.Node(orc_rules[root], [OF.Node(orc_rules[c], [None] * orc_rules[c].R) for c in children])


def dalberto():
    """Two levels of Strassen with the variant at products 1, 3, 4 (1-based)."""
    return ["S", ["D" if r in (0, 2, 3) else "S" for r in range(7)]]


def fast323_nonuniform():
    """Two levels of <3,2,3;15> with the permuted variants at the products
    the Sec. 3.4 example lists (1-based): F at 2, 6, 8, 14, 15; F1 at 1, 3,
    10, 11; F2 at 4, 5, 7, 9, 12, 13."""
    lab = {}
    lab.update({n: "F" for n in (2, 6, 8, 14, 15)})
    lab.update({n: "F1" for n in (1, 3, 10, 11)})
    lab.update({n: "F2" for n in (4, 5, 7, 9, 12, 13)})
    return ["F", [lab[r + 1] for r in range(15)]]


def mixed_rank():
    """Strassen at the root, classical <2,2,2;8> under products 2 and 5,
    Winograd elsewhere: the ranks of level 2 differ."""
    return ["S", ["C222" if r in (1, 4) else "Wg" for r in range(7)]]


def max_terms(orc):
    """Largest number of flattened terms of one leaf on any side (a bound:
    the product along each path of the per-rule maxima)."""
    if orc is None:
        return 1
    r = orc.rule
    p = OR.principal(r)
    here = int(max(p.alpha.max(), p.beta.max(), (r.W != 0).sum(axis=0).max()))
    return here * max(max_terms(c) for c in orc.children)


def uneven_delta():
    """Winograd at the root, Winograd under its second product (which adds
    into C block c11 alone, the block with the fewest terms) and classical
    <2,2,2;8> under the others: the largest delta_k of Sec. 4.5 is not the
    largest gamma_k plus the largest child delta."""
    return ["Wg", ["Wg" if r == 1 else "C222" for r in range(7)]]
