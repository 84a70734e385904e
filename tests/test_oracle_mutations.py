"""Plant plausible mistakes in copies of the oracle's C source and require
that each one fails at least one pin (CPU only; nothing here touches the
product library or a GPU)."""
import os
import shutil
import tempfile

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "fei_oracle.c")

# (name, [(exact text in the oracle, replacement), ...])
MUTATIONS = [
    ("drop_convection", [("A[(size_t)i * nsh + j] += s * (diff + phi[i] * conv + c * phi[i] * phi[j]);",
                          "A[(size_t)i * nsh + j] += s * (diff + c * phi[i] * phi[j]);")]),
    ("convection_sign", [("s * (diff + phi[i] * conv + c", "s * (diff - phi[i] * conv + c")]),
    ("convection_transposed", [("conv += bb[k] * gx[3 * j + k];", "conv += bb[k] * gx[3 * i + k];"),
                               ("s * (diff + phi[i] * conv + c", "s * (diff + phi[j] * conv + c")]),
    ("inverse_not_transposed", [("for (int l = 0; l < 3; ++l) s += R[l][k] * dphi[3 * j + l];\n        gx[3 * j + k] = s;\n      }\n    int64_t r = coef_index(B, e, q, nq);\n    const double *K = B->K + 9 * r, *bb = B->b + 3 * r;\n    double c = B->c[r], f = B->f[r];\n    double s = w * det;\n    /* steps",
                                 "for (int l = 0; l < 3; ++l) s += R[k][l] * dphi[3 * j + l];\n        gx[3 * j + k] = s;\n      }\n    int64_t r = coef_index(B, e, q, nq);\n    const double *K = B->K + 9 * r, *bb = B->b + 3 * r;\n    double c = B->c[r], f = B->f[r];\n    double s = w * det;\n    /* steps")]),
    ("K_transposed", [("diff += gx[3 * i + k] * K[3 * k + l] * gx[3 * j + l];",
                       "diff += gx[3 * i + k] * K[3 * l + k] * gx[3 * j + l];")]),
    ("reaction_dropped", [("s * (diff + phi[i] * conv + c * phi[i] * phi[j]);", "s * (diff + phi[i] * conv);")]),
    ("load_missing_det", [("bv[i] += s * f * phi[i];", "bv[i] += w * f * phi[i];")]),
    ("duffy_weight", [("(1.0 - v) / 8.0", "(1.0 - v) / 4.0")]),
    ("duffy_map", [("pts[4 * q + 0] = 0.25 * (1.0 + u) * (1.0 - v);", "pts[4 * q + 0] = 0.25 * (1.0 + u) * (1.0 + v);")]),
    ("gauss_weight", [("w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);", "w[n - 1 - i] = 2.0 / ((1.0 + t * t) * dP * dP);")]),
    ("jacobi_alpha", [("double Q = jacobi(n, 2.0 * m + 1.0, 0.0, eta2);", "double Q = jacobi(n, 2.0 * m, 0.0, eta2);")]),
    ("dubiner_norm", [("double c = sqrt(2.0 * (2.0 * m + 1.0) * (m + n + 1.0));", "double c = sqrt(2.0 * (2.0 * m + 1.0) * (m + n + 2.0));")]),
    ("dubiner_deriv_sign", [("A * (-(double)m * om_m1 * Q + 2.0 * om_m * dQ)", "A * ((double)m * om_m1 * Q + 2.0 * om_m * dQ)")]),
    ("legendre_norm", [("double s = sqrt((2.0 * k + 1.0) / 2.0);", "double s = sqrt((2.0 * k + 1.0));")]),
    ("legendre_deriv", [("double d2 = d0 + (2.0 * k + 1.0) * p1;", "double d2 = d0 + (2.0 * k) * p1;")]),
    ("vertex_grad_sign", [("g[a][2] = -0.5 * lam[a];", "g[a][2] = 0.5 * lam[a];")]),
    ("det_cofactor_sign", [("J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +", "J[0][1] * (J[1][0] * J[2][2] + J[1][2] * J[2][0]) +")]),
    ("inverse_entry", [("R[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;", "R[1][2] = (J[0][0] * J[1][2] - J[0][2] * J[1][0]) / d;")]),
    ("bwd_drop_conv_grad", [("gP[3 * j + k] += s * a * phi[i] * bb[k];", "")]),
    ("bwd_inverse_sign", [("gJ[k][l] = gs * s * R[l][k] - t;", "gJ[k][l] = gs * s * R[l][k] + t;")]),
    ("bwd_det_transposed", [("gJ[k][l] = gs * s * R[l][k] - t;", "gJ[k][l] = gs * s * R[k][l] - t;")]),
    ("bwd_K_grad_transposed", [("for (int l = 0; l < 3; ++l) gK[k][l] += a * Pi[k] * Pj[l];",
                                "for (int l = 0; l < 3; ++l) gK[k][l] += a * Pi[l] * Pj[k];")]),
    ("bwd_missing_load_in_gs", [("gs += gb[i] * f * phi[i];", "")]),
]


def _run_pins():
    failed = []
    for name, fn in P.ALL_PINS:
        try:
            fn()
        except AssertionError:
            failed.append(name)
        except Exception as exc:  # a crash of a broken build also counts as caught
            failed.append(f"{name}:{type(exc).__name__}")
    return failed


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="fei_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,subs", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(name, subs, workdir):
    with open(SRC) as fh:
        text = fh.read()
    for old, new in subs:
        assert text.count(old) == 1, f"mutation anchor not unique/found: {old[:60]}"
        text = text.replace(old, new)
    src = os.path.join(workdir, f"{name}.c")
    with open(src, "w") as fh:
        fh.write(text)
    lib = oracle.compile_source(src, os.path.join(workdir, f"lib_{name}.so"))
    oracle.use_library(lib)
    try:
        failed = _run_pins()
    finally:
        oracle.use_library(None)
    assert failed, f"mutation {name} passed every pin"
