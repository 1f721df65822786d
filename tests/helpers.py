"""Small helpers shared by the tests (no solver arithmetic)."""
import numpy as np


def half_ulp_of_printed(s):
    """Half a unit in the last printed digit of a decimal string."""
    s = s.strip().lstrip("+-")
    if "." in s:
        return 0.5 * 10.0 ** (-(len(s.split(".")[1])))
    return 0.5


def read_golden(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def mirror_x(u):
    """Mirror a conserved state [5, nz, ny, nx] in x (flip x, negate x momentum)."""
    m = u[:, :, :, ::-1].copy()
    m[1] = -m[1]
    return m


def rotate_xyz(u):
    """Cyclic axis permutation x->y->z->x of a conserved state [5, nz, ny, nx].

    The new field at (z', y', x') = (y, x, z) ... i.e. the old x axis becomes
    the new y axis, old y becomes new z, old z becomes new x; momentum
    components move with their axes.
    """
    # old array axes (z, y, x) -> new array axes (z'=old y, y'=old x, x'=old z)
    r = np.transpose(u, (0, 2, 3, 1)).copy()
    out = r.copy()
    out[1] = r[3]  # new x momentum = old z momentum
    out[2] = r[1]  # new y momentum = old x momentum
    out[3] = r[2]  # new z momentum = old y momentum
    return out


def build_oracle_mutant(tag, edits):
    """Compile a copy of the oracle with planted mistakes and load it.

    ``edits`` is a list of (function_head, old, new): inside the function whose
    definition starts with ``function_head`` (up to its closing brace at column
    0), the text ``old`` -- which must occur there exactly once -- is replaced
    by ``new``.  The copy is compiled with the oracle's own flags into a
    temporary directory; returns the loaded ``ctypes.CDLL``.  Used to check that
    a pin fails when the oracle is wrong.
    """
    import ctypes
    import os
    import subprocess
    import tempfile

    from oracle import build_oracle

    with open(build_oracle.SRC) as f:
        src = f.read()
    for head, old, new in edits:
        a = src.index(head)
        b = src.index("\n}\n", a) + 3
        body = src[a:b]
        assert body.count(old) == 1, (tag, head, old, body.count(old))
        src = src[:a] + body.replace(old, new) + src[b:]
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    path_c = os.path.join(d, "mutant_%s.cpp" % tag)
    path_so = os.path.join(d, "libmutant_%s.so" % tag)
    with open(path_c, "w") as f:
        f.write(src)
    subprocess.run(["g++"] + build_oracle.FLAGS + [path_c, "-o", path_so], check=True)
    return ctypes.CDLL(path_so)
