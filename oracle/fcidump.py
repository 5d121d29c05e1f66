"""FCIDUMP reader and writer (oracle, test infrastructure only).

The paper's molecular integrals are not available; a user who has real ones
supplies them in the common FCIDUMP text form: a Fortran namelist header
``&FCI NORB=n, NELEC=ne, MS2=m, ... &END`` (or ``/``), then one line per
integral, ``value i j k l`` with 1-based orbital indices:

* i, j, k, l all non-zero: the chemist two-electron integral (ij|kl);
* k = l = 0, i, j non-zero: the one-electron integral h_ij;
* all zero: the core (constant) energy;
* any other pattern (orbital energies): ignored.

Real orbitals: (ij|kl) has the 8-fold symmetry (ij|kl) = (ji|kl) =
(ij|lk) = (kl|ij) and h is symmetric, so a file may list each class once.
Values may use a Fortran ``D`` exponent.
"""

import re

import numpy as np


def _header_value(text, key):
    m = re.search(r"\b" + key + r"\s*=\s*(-?\d+)", text, re.IGNORECASE)
    return int(m.group(1)) if m else None


def read(path):
    """(h[n, n], g[n, n, n, n], e_core, norb, nelec, ms2) from a FCIDUMP file."""
    text = open(path).read()
    m = re.search(r"(&END|/)", text[text.upper().index("&FCI"):], re.IGNORECASE)
    cut = text.upper().index("&FCI") + m.end()
    header, body = text[:cut], text[cut:]
    n = _header_value(header, "NORB")
    ne = _header_value(header, "NELEC")
    ms2 = _header_value(header, "MS2") or 0
    h = np.zeros((n, n))
    g = np.zeros((n, n, n, n))
    e = 0.0
    tok = body.replace("D", "E").replace("d", "e").split()
    for t in range(0, len(tok) - len(tok) % 5, 5):
        v = float(tok[t])
        i, j, k, l = (int(x) for x in tok[t + 1:t + 5])
        if i and j and k and l:
            i, j, k, l = i - 1, j - 1, k - 1, l - 1
            for a, b, c, d in ((i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                               (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)):
                g[a, b, c, d] = v
        elif i and j and not k and not l:
            h[i - 1, j - 1] = v
            h[j - 1, i - 1] = v
        elif not (i or j or k or l):
            e = v
    return h, g, e, n, ne, ms2


def write(path, h, g, e_core, nelec, ms2=0, tol=0.0):
    """Write the symmetry-unique integrals with |v| > tol (i >= j, k >= l,
    ij >= kl for g; i >= j for h), then the core energy."""
    n = h.shape[0]
    lines = [f" &FCI NORB={n},NELEC={nelec},MS2={ms2},", "  ORBSYM=" + ",".join("1" * n) + ",",
             "  ISYM=1,", " &END"]
    for i in range(n):
        for j in range(i + 1):
            for k in range(n):
                for l in range(k + 1):
                    if i * (i + 1) // 2 + j < k * (k + 1) // 2 + l:
                        continue
                    v = g[i, j, k, l]
                    if abs(v) > tol:
                        lines.append(f"{v: .16E} {i + 1:4d} {j + 1:4d} {k + 1:4d} {l + 1:4d}")
    for i in range(n):
        for j in range(i + 1):
            if abs(h[i, j]) > tol:
                lines.append(f"{h[i, j]: .16E} {i + 1:4d} {j + 1:4d}    0    0")
    lines.append(f"{e_core: .16E}    0    0    0    0")
    open(path, "w").write("\n".join(lines) + "\n")
