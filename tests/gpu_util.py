"""Helpers for the GPU parity tests (no test functions here)."""

import numpy as np

import paper_2606_29692_gb300 as tq


class _DevArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def dev_to_numpy(ptr, n, typestr):
    """Copy ``n`` elements at device pointer ``ptr`` into a numpy array."""
    import torch
    if n == 0:
        return np.zeros(0, dtype=np.dtype(typestr))
    t = torch.as_tensor(_DevArray(ptr, n, typestr), device="cuda")
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def ham_csr_numpy(ham):
    """(rowptr, col, val, diag) of a device Hamiltonian as numpy arrays."""
    rp, cl, vl, dg = tq.ham_csr(ham)
    D = getattr(ham, "dim", 1 << ham.n_qubits)
    rowptr = dev_to_numpy(rp, D + 1, "<i4")
    nnz = int(rowptr[-1])
    col = dev_to_numpy(cl, nnz, "<i4")
    val = dev_to_numpy(vl, nnz, "<f8" if ham.prec == tq.TQ_C128 else "<f4")
    diag = dev_to_numpy(dg, D, "<f8")
    return rowptr, col, val, diag


def oracle_split(H):
    """Oracle CSR split into (rowptr, col, val) of the off-diagonal part and diag."""
    H = H.tocsr()
    H.sort_indices()
    D = H.shape[0]
    diag = H.diagonal().real.copy()
    coo = H.tocoo()
    off = coo.row != coo.col
    r, c, v = coo.row[off], coo.col[off], coo.data[off].real
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr), c, v, diag


def to_state(ctx, psi, nq, prec, sector=None):
    import torch
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    t = torch.as_tensor(np.asarray(psi), dtype=dt).to("cuda").contiguous()
    return tq.State(ctx, nq, prec, tensor=t, sector=sector)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fidelity(a, b):
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))
