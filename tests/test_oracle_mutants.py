"""The pins catch plausible mistakes: each case plants one mistake in a copy
of ph_oracle.c (built in a temporary directory, the oracle itself is not
touched), and at least one pin must fail on it."""
import math
import os
import subprocess

import numpy as np
import pytest

import meshgen
import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "ph_oracle.c")
REF = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)

MUTANTS = {
    "K prefactor |T|/6": ("g->K[i][j] = g->vol * s;", "g->K[i][j] = g->vol / 6 * s;"),
    "mass diagonal": ("g->M[i][j] = g->vol / 20 * ((i == j) ? 2 : 1);", "g->M[i][j] = g->vol / 20 * ((i == j) ? 1 : 1);"),
    "area factor": ("g->area[k] = qsqrt(cx * cx + cy * cy + cz * cz) / 2;",
                    "g->area[k] = qsqrt(cx * cx + cy * cy + cz * cz) / 3;"),
    "C entries 1/3": ("qf val = on_face(k, j) ? (qf)sig4[k] * G->area[k] / 3 : 0;",
                      "qf val = on_face(k, j) ? (qf)sig4[k] * G->area[k] / 4 : 0;"),
    "C transposed": ("for (int k = 0; k < 4; ++k) R[j][k] = L.C[k][j]; /* C' */",
                     "for (int k = 0; k < 4; ++k) R[j][k] = L.C[j][k]; /* C' */"),
    "load weight": ("s += (qf)f4[k] / 3;", "s += (qf)f4[k] / 4;"),
    "rhs sign": ("g_out[k] = (double)(-s);", "g_out[k] = (double)(s);"),
    "sigma dropped in assembly": ("sig[k] = (tf < 0) ? -1 : 1;\n    kind[k] = face_kind[F];\n    mult[k] = face_mult[F];",
                                  "sig[k] = 1;\n    kind[k] = face_kind[F];\n    mult[k] = face_mult[F];"),
    "b_D sign": ("rhs[face_mult[F]] += bD;", "rhs[face_mult[F]] -= bD;"),
    "recovery sign": ("for (int k = 0; k < 4; ++k) s += Lq.C[k][j] * lam[k];",
                      "for (int k = 0; k < 4; ++k) s -= Lq.C[k][j] * lam[k];"),
    "local face order": ("{{0, 1, 2}, {0, 2, 3}, {0, 3, 1}, {3, 2, 1}}", "{{0, 1, 2}, {0, 2, 3}, {0, 3, 1}, {1, 2, 3}}"),
    "T+ is the later tet": ("if (nt == 0) s0 = rec[l].slot; else if (nt == 1) s1 = rec[l].slot;",
                            "if (nt == 0) s1 = rec[l].slot; else if (nt == 1) s0 = rec[l].slot;"),
    "reaction dropped": ("L->A[i][j] = (qf)a * G->K[i][j] + (qf)c * G->M[i][j];",
                         "L->A[i][j] = (qf)a * G->K[i][j] + (qf)c * G->M[i][j] * (i == j);"),
}


def pins():
    """Each returns True when the pin holds."""

    def closed_form():
        S, _ = oracle.tet_local(REF, 1.0, 1.0, [0, 0, 0, 0], [1, 1, 1, 1])
        want = np.array([8212 / 5103, 7402 / 5103, 362 * math.sqrt(3) / 243, 124 / 27])
        got = np.array([S[0, 0], S[0, 1], S[0, 3], S[3, 3]])
        return np.allclose(got, want, rtol=1e-14, atol=0)

    def textbook_matrices():
        m = oracle.tet_matrices(REF)
        K = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6
        return (np.allclose(m["K"], K, atol=1e-16) and np.allclose(m["M"], (np.eye(4) + 1) / 120, atol=1e-18)
                and np.allclose(m["area"], [0.5, 0.5, 0.5, math.sqrt(3) / 2], rtol=1e-15))

    def constant_load():
        P = REF + np.array([[0.1, 0.2, 0.0], [0.3, 0.0, 0.1], [0.0, 0.0, 0.2], [0.1, 0.1, 0.1]])
        sig = np.array([1, -1, 1, -1])
        _, g = oracle.tet_local(P, 2.0, 0.5, [3.0] * 4, sig)
        area = oracle.tet_matrices(P)["area"]
        return np.allclose(g, -(3.0 / 0.5) * sig * area, rtol=1e-13)

    def faces_example():
        coord, tet, _, _ = meshgen.listing1_mesh()
        fc = oracle.faces(tet, 8)
        LF = [(0, 1, 2), (0, 2, 3), (0, 3, 1), (3, 2, 1)]
        ok = fc["nF"] == 16 and [(int(x) & 0x7FFFFFFF) + 1 for x in fc["tet_face"][4]] == [16, 7, 12, 4]
        ok = ok and all(int(x) < 0 for x in fc["tet_face"][4])
        for t in range(4):
            for k in range(4):
                ok = ok and list(fc["face_vtx"][4 * t + k]) == [tet[t][j] for j in LF[k]]
        return bool(ok)

    def monolithic():
        from tests.test_oracle_system import test_condensed_equals_monolithic
        try:
            test_condensed_equals_monolithic("mixed1")
            test_condensed_equals_monolithic("kuhn_lognormal")
            return True
        except AssertionError:
            return False

    def patch():
        from tests.test_oracle_system import test_patch_constant
        try:
            test_patch_constant()
            return True
        except AssertionError:
            return False

    return {"closed_form": closed_form, "textbook": textbook_matrices, "constant_load": constant_load,
            "faces_example": faces_example, "monolithic": monolithic, "patch": patch}


def test_every_pin_holds_on_the_oracle():
    for name, pin in pins().items():
        assert pin(), name


def run_pins_with(so_path):
    """Names of the pins that fail on the library at so_path."""
    failed = []
    with oracle.use_library(so_path):
        for pin_name, pin in pins().items():
            try:
                ok = pin()
            except Exception:
                ok = False
            if not ok:
                failed.append(pin_name)
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    import json
    import sys
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not found: {old}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", str(path), "-o", str(so), "-lm"])
    # a separate process: a mutant may also corrupt memory and crash, which counts as caught
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import json, sys; sys.path.insert(0, %r); from tests.test_oracle_mutants import run_pins_with; "
            "print(json.dumps(run_pins_with(%r)))" % (root, str(so)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return  # crashed on the mutant: caught
    failed = json.loads(r.stdout.strip().splitlines()[-1])
    assert failed, f"mutant '{name}' passes every pin"
