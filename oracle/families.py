"""Commuting-family partition of the pool (Sec. III-F, Algorithm 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The pool is split into families of mutually commuting generators by a
greedy colouring of the non-commutativity graph.  The paper names the
relation two ways: operators that "share qubit-wise commuting components"
(Sec. III-B) and operators with [A_i, A_j] = 0 (Sec. III-F).  Both are
offered:

* ``FULL``: an edge joins i and j when the commutator A_i A_j - A_j A_i is
  not the zero operator (computed here from dense matrices);
* ``QWC``: an edge joins i and j unless every Pauli string of A_i commutes
  qubit-wise with every Pauli string of A_j (on each qubit the two letters
  are equal or one is the identity).

Colouring, in the order Algorithm 1 gives: vertices sorted by descending
degree (ties by ascending pool index: a stable sort), each vertex joins the
lowest-indexed family holding none of its neighbours, else opens a new
family.
"""

import numpy as np

FULL = 0
QWC = 1


def full_edges(pool_matrices):
    """Pairs (i, j), i < j, whose dense matrices do not commute."""
    mats = [A.toarray() if hasattr(A, "toarray") else np.asarray(A) for A in pool_matrices]
    edges = set()
    for i in range(len(mats)):
        for j in range(i + 1, len(mats)):
            comm = mats[i] @ mats[j] - mats[j] @ mats[i]
            if np.abs(comm).max() > 1e-12:
                edges.add((i, j))
    return edges


def labels(ps):
    """Pauli labels (qubit 0 first) of a Pauli sum's terms, from its X and Z masks."""
    out = []
    for x, z in zip(ps.x, ps.z):
        out.append("".join("IXZY"[((int(x) >> q) & 1) | (((int(z) >> q) & 1) << 1)] for q in range(ps.n_qubits)))
    return out


def qubit_wise_commute(label_a, label_b):
    """Two Pauli labels (strings over I, X, Y, Z) commute qubit-wise."""
    return all(a == "I" or b == "I" or a == b for a, b in zip(label_a, label_b))


def qwc_edges(pool_labels):
    """Pairs (i, j), i < j, with some term pair that is not qubit-wise commuting.

    ``pool_labels[k]`` lists the Pauli labels of generator k's terms."""
    edges = set()
    for i in range(len(pool_labels)):
        for j in range(i + 1, len(pool_labels)):
            if not all(qubit_wise_commute(a, b) for a in pool_labels[i] for b in pool_labels[j]):
                edges.add((i, j))
    return edges


def greedy_families(n, edges):
    """Algorithm 1: largest-first greedy colouring.  Returns family[v]."""
    nbr = [set() for _ in range(n)]
    for i, j in edges:
        nbr[i].add(j)
        nbr[j].add(i)
    order = sorted(range(n), key=lambda v: -len(nbr[v]))      # stable: ties by index
    family = [-1] * n
    members = []                                                # family -> set of vertices
    for v in order:
        for f, mem in enumerate(members):
            if not (nbr[v] & mem):
                family[v] = f
                mem.add(v)
                break
        else:
            family[v] = len(members)
            members.append({v})
    return family


def family_order(family):
    """Pool indices laid out family by family (ascending index inside a family)."""
    return sorted(range(len(family)), key=lambda v: (family[v], v))
