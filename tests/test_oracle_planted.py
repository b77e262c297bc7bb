"""Planted mistakes: the oracle's pins must reject a wrong oracle.

Each case copies ``oracle/sem_oracle.c``, plants one plausible mistake in the
copy (a dropped term, a wrong sign, index or factor, a transposed operand, a
missing weight), compiles it with the oracle's own flags and runs the pin
tests that cover that function against it (``SEM_ORACLE_LIB``).  The pins
must fail.  The unaltered copy, built and loaded the same way, must pass, so
the failures come from the planted mistakes and not from the harness.  The
copies are built and run in parallel, each test process on one thread, and
the pins marked slow (larger meshes of the same checks) are left out.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sem_oracle.c")

BASIS = "tests/test_oracle_basis.py"
OPER = "tests/test_oracle_operator.py"
SOLV = "tests/test_oracle_solvers.py"
ASM = "tests/test_oracle_schwarz.py"

# (name, text in the oracle, planted replacement, pin files that must fail)
PLANTED = [
    ("gll weights lose the square of P_N",
     "w[i] = 2.0 / (N * (N + 1.0) * p * p);", "w[i] = 2.0 / (N * (N + 1.0) * p);", [BASIS]),
    ("Dhat stored transposed",
     "D[i * (N + 1) + l] = lagrange_deriv(N, xi, l, xi[i]);",
     "D[l * (N + 1) + i] = lagrange_deriv(N, xi, l, xi[i]);", [BASIS, OPER]),
    ("interpolation evaluated at the mirrored fine nodes",
     "J[i * (Nc + 1) + j] = lagrange(Nc, xc, j, xf[i]);",
     "J[i * (Nc + 1) + j] = lagrange(Nc, xc, j, xf[Nf - i]);", [BASIS]),
    ("adjugate entry with the wrong sign",
     "Inv[0][1] = (Jac[0][2] * Jac[2][1] - Jac[0][1] * Jac[2][2]) / det;",
     "Inv[0][1] = (Jac[0][1] * Jac[2][2] - Jac[0][2] * Jac[2][1]) / det;", [BASIS, OPER]),
    ("factors rs and rt swapped",
     "ee[6] = {0, 1, 2, 1, 2, 2};", "ee[6] = {0, 2, 1, 1, 2, 2};", [BASIS, OPER]),
    ("quadrature weight index k written as j",
     "double W = w[i] * w[j] * w[k] * det;", "double W = w[i] * w[j] * w[j] * det;",
     [BASIS, OPER]),
    ("global ids with the x stride for y planes",
     "ids[e * Np * Np * Np + i + Np * (j + Np * k)] = gx + nx * (gy + ny * gz);",
     "ids[e * Np * Np * Np + i + Np * (j + Np * k)] = gx + nx * (gy + nx * gz);",
     [BASIS, OPER]),
    ("t-direction divergence term dropped",
     "            s += D[l * Np + k] * ut[i + Np * (j + Np * l)];\n", "", [OPER]),
    ("flux u_s mixes with G_rt instead of G_rs",
     "us[p] = Grs * a + Gss * b + Gst * c;", "us[p] = Grt * a + Gss * b + Gst * c;", [OPER]),
    ("divergence applies Dhat instead of its transpose",
     "s += D[l * Np + i] * ur[l + Np * (j + Np * k)];",
     "s += D[i * Np + l] * ur[l + Np * (j + Np * k)];", [OPER]),
    ("gather-scatter overwrites instead of summing",
     "for (int64_t l = 0; l < nl; ++l) acc[ids[l]] += u[l];",
     "for (int64_t l = 0; l < nl; ++l) acc[ids[l]] = u[l];", [BASIS, OPER]),
    ("inner product without the 1/multiplicity weight",
     "s += u[l] * v[l] * L->inv_mult[l];", "s += u[l] * v[l];", [OPER, SOLV]),
    ("diagonal cross term without its factor 2",
     "s += 2.0 * Di * Dj * g[1 * Np3 + p];", "s += Di * Dj * g[1 * Np3 + p];", [OPER, SOLV]),
    ("Chebyshev recurrence with rho for rho'",
     "d[l] = rho1 * rho * d[l] + (2.0 * rho1 / delta) * dinv[l] * r[l];",
     "d[l] = rho1 * rho * d[l] + (2.0 * rho / delta) * dinv[l] * r[l];", [SOLV]),
    ("Lanczos diagonal divides by the wrong alpha",
     "ta[j] = 1.0 / alph[j] + (j > 0 ? bet[j - 1] / alph[j - 1] : 0.0);",
     "ta[j] = 1.0 / alph[j] + (j > 0 ? bet[j - 1] / alph[j] : 0.0);", [SOLV]),
    ("splitmix64 with the wrong first shift",
     "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;",
     [BASIS]),
    ("restriction without the transpose",
     "double Ja = transpose ? J[a * nc + i] : J[i * nc + a];",
     "double Ja = transpose ? J[i * nc + a] : J[i * nc + a];", [SOLV]),
    ("restriction without the 1/multiplicity weight",
     "  for (int64_t i = 0; i < n; ++i) r[i] *= L->inv_mult[i];\n", "", [SOLV]),
    ("V-cycle without post-smoothing",
     "orc_cheb(n, level_apply, L, L->dinv, b, x, P->cheb_degree, L->lam_lo, L->lam_hi, 0);",
     "(void)0;", [SOLV]),
    ("FlexCG with the Fletcher-Reeves coefficient",
     "double beta = (zr - zro) / rho;", "double beta = zr / rho;", [SOLV]),
    ("FGMRES with every Gram-Schmidt coefficient against v_0",
     "H[i * m + j] = orc_level_dot(L, w, V + (size_t)i * n);",
     "H[i * m + j] = orc_level_dot(L, w, V);", [SOLV]),
    ("FGMRES Givens rotation with the wrong sign",
     "g[j + 1] = -sn[j] * g[j];", "g[j + 1] = sn[j] * g[j];", [SOLV]),
    ("projection norm without the Pythagoras correction",
     "  for (int i = 0; i < k; ++i) nrm2 -= alpha[i] * alpha[i];\n", "", [SOLV]),
    ("Schwarz 1D mass with h inverted",
     "B[(i + 1) * n + (i + 1)] += 0.5 * he * L->w[i];",
     "B[(i + 1) * n + (i + 1)] += 0.5 / he * L->w[i];", [ASM]),
    ("Schwarz left neighbour points in the wrong order",
     "int li[2] = {N - 1, N}, ai[2] = {0, 1};", "int li[2] = {N, N - 1}, ai[2] = {0, 1};", [ASM]),
    ("Legendre derivative recurrence from the wrong term",
     "double d2 = d0 + (2.0 * k + 1.0) * p1;", "double d2 = d1 + (2.0 * k + 1.0) * p1;", [BASIS]),
    ("Newton step with the wrong sign in Legendre's equation",
     "double d2p = (2.0 * x * dp - N * (N + 1.0) * p) / (1.0 - x * x);",
     "double d2p = (2.0 * x * dp + N * (N + 1.0) * p) / (1.0 - x * x);", [BASIS]),
    ("Dirichlet mask misses the bottom face",
     "int onb = gx == 0 || gy == 0 || gz == 0 ||", "int onb = gx == 0 || gy == 0 ||",
     [BASIS, OPER, SOLV]),
    ("Jacobi diagonal not inverted",
     "L->dinv[l] = L->mask[l] / L->dinv[l];", "L->dinv[l] = L->mask[l] * L->dinv[l];",
     [OPER, SOLV]),
    ("multiplicity never summed",
     "  orc_gs(L->nl, L->ids, L->ng, L->mult);\n", "", [BASIS, OPER, SOLV]),
    ("prolongation with a for b in the second factor",
     "double Jb = transpose ? J[b * nc + j] : J[j * nc + b];",
     "double Jb = transpose ? J[b * nc + j] : J[j * nc + a];", [SOLV]),
    ("Lanczos start vector keeps its mean under Neumann",
     "for (int64_t l = 0; l < n; ++l) v[l] -= s / c;", "(void)s;", [SOLV, ASM]),
    ("tridiagonal bisection keeps the lowest eigenvalue",
     "if (cnt == m) hi = mid; else lo = mid;", "if (cnt >= 1) hi = mid; else lo = mid;",
     [SOLV, ASM]),
    ("Schwarz extension takes the shared face point",
     "idx[out] = N - 1;", "idx[out] = N;", [ASM]),
    ("Schwarz local matrix with A for B in x",
     "B[2][c * n + c2] * A[1][b * n + b2] * B[0][a * n + a2] +",
     "B[2][c * n + c2] * A[1][b * n + b2] * A[0][a * n + a2] +", [ASM]),
    ("Chebyshev on M A starts with delta for theta",
     "for (int64_t l = 0; l < n; ++l) d[l] = mr[l] / theta;",
     "for (int64_t l = 0; l < n; ++l) d[l] = mr[l] / delta;", [ASM, SOLV]),
    ("FGMRES back substitution adds instead of subtracting",
     "for (int q = i + 1; q < cols; ++q) s -= H[i * m + q] * y[q];",
     "for (int q = i + 1; q < cols; ++q) s += H[i * m + q] * y[q];", [SOLV]),
    ("projected solve forgets the best fit",
     "    x[l] = xb;", "    x[l] = 0.0 * xb;", [SOLV]),
    ("PCG initial residual with the wrong sign of A x0",
     "  for (int64_t l = 0; l < n; ++l) r[l] = b[l] - w[l];\n  double bnorm = sqrt(orc_level_dot(L, b, b));\n"
     "  double rnorm = sqrt(orc_level_dot(L, r, r));\n  *res0 = rnorm;\n  int k = 0, status = 1;\n"
     "  if (rnorm <= tol * bnorm || rnorm == 0.0) status = 0;\n  if (status != 0) {\n"
     "    for (int64_t l = 0; l < n; ++l) z[l] = (precond",
     "  for (int64_t l = 0; l < n; ++l) r[l] = b[l] + w[l];\n  double bnorm = sqrt(orc_level_dot(L, b, b));\n"
     "  double rnorm = sqrt(orc_level_dot(L, r, r));\n  *res0 = rnorm;\n  int k = 0, status = 1;\n"
     "  if (rnorm <= tol * bnorm || rnorm == 0.0) status = 0;\n  if (status != 0) {\n"
     "    for (int64_t l = 0; l < n; ++l) z[l] = (precond", [SOLV]),
    ("Schwarz forward substitution reads the upper triangle",
     "for (int k = 0; k < i; ++k) s -= C[(size_t)i * n3 + k] * u[k];",
     "for (int k = 0; k < i; ++k) s -= C[(size_t)k * n3 + i] * u[k];", [ASM]),
    ("Schwarz element length as half the sum of four edges",
     "h[e * 3 + d] = 0.25 * s;", "h[e * 3 + d] = 0.5 * s;", [ASM]),
    ("Schwarz right extension takes the shared face point",
     "idx[out] = 1;", "idx[out] = 0;", [ASM]),
    ("GLL Newton started from the mirrored guesses",
     "double x = -cos(ORC_PI * i / N);", "double x = cos(ORC_PI * i / N);", [BASIS]),
    ("prolongation stored transposed",
     "ve[i + no * (j + no * k)] = s;", "ve[k + no * (j + no * i)] = s;", [SOLV]),
    ("diagonal s-term with G_rr",
     "s += D[l * Np + j] * D[l * Np + j] * g[3 * Np3 + i + Np * (l + Np * k)];",
     "s += D[l * Np + j] * D[l * Np + j] * g[0 * Np3 + i + Np * (l + Np * k)];", [OPER, SOLV]),
    ("FlexCG keeps the new residual as the old one",
     "{ rold[l] = r[l]; r[l] -= alpha * w[l]; }", "{ r[l] -= alpha * w[l]; rold[l] = r[l]; }",
     [SOLV]),
    ("FGMRES first basis vector not normalised",
     "for (int64_t l = 0; l < n; ++l) V[l] /= beta;", "(void)0;", [SOLV]),
    ("projection coefficients against A p_i",
     "for (int i = 0; i < k; ++i) c[i] = orc_level_dot(L, Q->P + (size_t)i * n, b);",
     "for (int i = 0; i < k; ++i) c[i] = orc_level_dot(L, Q->AP + (size_t)i * n, b);", [SOLV]),
    ("Lanczos off-diagonal without the square root",
     "if (j < k - 1) tb[j] = sqrt(bet[j]) / alph[j];", "if (j < k - 1) tb[j] = bet[j] / alph[j];",
     [SOLV, ASM]),
    ("Dirichlet mask applied under Neumann too",
     "(bc == 0 && onb) ? 0.0 : 1.0;", "(onb) ? 0.0 : 1.0;", [BASIS, OPER, SOLV]),
    ("geometry interpolates x with l_b for l_c",
     "x[m] += Xv * lr[a] * ls[b] * lt[c];", "x[m] += Xv * lr[a] * ls[b] * lt[b];", [BASIS, OPER]),
]


def _build_and_run(src_text, out_dir, files):
    import oracle

    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "sem_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    so = oracle.compile_to(src, os.path.join(out_dir, "libsemoracle.so"))
    env = dict(os.environ, SEM_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-m", "pytest", *files, "-x", "-q", "-m",
                        "not gpu and not slow",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return p.returncode, p.stdout[-2000:] + p.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    import oracle

    oracle.build()
    text = open(SRC).read()
    jobs = [("unaltered", text, [BASIS, OPER, SOLV, ASM])]
    for name, old, new, files in PLANTED:
        assert text.count(old) == 1, f"{name}: the planted site must occur once"
        jobs.append((name, text.replace(old, new), files))
    root = tmp_path_factory.mktemp("planted")
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = {name: ex.submit(_build_and_run, t, str(root / f"m{i}"), files)
                for i, (name, t, files) in enumerate(jobs)}
        return {name: f.result() for name, f in futs.items()}


def test_unaltered_oracle_passes_through_the_harness(outcomes):
    rc, out = outcomes["unaltered"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [p[0] for p in PLANTED])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    # 1 = tests ran and some failed (not a collection or usage error)
    assert rc == 1 and "failed" in out, out
