"""Planted mistakes in the oracle must fail its pins.

Every parity claim rests on the oracle, and the oracle rests on its pins
(tests/test_oracle_pins*.py).  Each case below copies the oracle package into
a scratch directory, plants one plausible mistake in that copy (a dropped
term, a flipped sign, a wrong index range, a transposed block, an
off-by-one), and runs the pins that should catch it against the copy in a
fresh interpreter.  The case passes when those pins fail (pytest exit code 1:
test failures, not a collection or import error).  The tree under test is
never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

P = "tests/test_oracle_pins.py::"
PT = "tests/test_oracle_pins_tree.py::"
PH = "tests/test_oracle_pins_helmholtz.py::"

# (case id, oracle file, function (or Class.method) whose body holds the text,
# original text, planted text, pins that must fail)
MUTATIONS = [
    ("self-term-constant", "kernels.py", "self_integral",
     "- 1.5 + 0.25 * math.pi", "+ 1.5 + 0.25 * math.pi",
     [P + "test_self_cell_2d_matches_quadrature"]),
    ("green-3d-factor", "kernels.py", "green",
     "return 1.0 / (FOUR_PI * r)", "return 1.0 / (TWO_PI * r)",
     [P + "test_green_functions_eq_1_4"]),
    ("operator-b-c-swapped", "kernels.py", "kernel_entries",
     "return self.b[rows][:, None] * K * self.c[cols][None, :]",
     "return self.c[rows][:, None] * K * self.b[cols][None, :]",
     [P + "test_operator_b_scales_rows_c_scales_columns"]),
    ("id-tie-highest-index", "idqr.py", "interp_decomp",
     "p = j + cand[np.argmin(perm[j + cand])]", "p = j + cand[np.argmax(perm[j + cand])]",
     [P + "test_id_tie_break_lowest_index"]),
    ("id-threshold-from-current-pivot", "idqr.py", "interp_decomp",
     "        if j == 0:\n            nu0 = best\n", "        nu0 = best\n",
     [P + "test_id_exact_low_rank", P + "test_id_bounds_eq_2_3"]),
    ("id-T-columns-unordered", "idqr.py", "interp_decomp",
     "    T = T[:, order]\n", "",
     [P + "test_id_exact_low_rank", P + "test_id_bounds_eq_2_3"]),
    ("B_rr-dropped-term", "hifie.py", "_skeletonize",
     "B_rr = A_rr - T.T @ A_sr - A_rs @ T + T.T @ A_ss @ T", "B_rr = A_rr - T.T @ A_sr - A_rs @ T",
     [P + "test_skeletonization_decouples_redundant_dofs_lemma_2_3"]),
    ("B_sr-sign", "hifie.py", "_skeletonize",
     "B_sr = A_sr - A_ss @ T", "B_sr = A_sr + A_ss @ T",
     [P + "test_skeletonization_decouples_redundant_dofs_lemma_2_3"]),
    ("schur-sign", "hifie.py", "_skeletonize",
     "delta = -B_sr @ np.linalg.solve(B_rr, B_rs)", "delta = B_sr @ np.linalg.solve(B_rr, B_rs)",
     [P + "test_nonsymmetric_accuracy_full_compression"]),
    ("proxy-in-rows-missing", "hifie.py", "_skeletonize",
     "YK = np.vstack([YK_near1, YK_near2, YK_out, YK_in])",
     "YK = np.vstack([YK_near1, YK_near2, YK_out, 0.0 * YK_in])",
     [P + "test_proxy_rows_span_far_field_lemma_3_3"]),
    ("proxy-out-rows-missing", "hifie.py", "_skeletonize",
     "YK = np.vstack([YK_near1, YK_out])", "YK = np.vstack([YK_near1, 0.0 * YK_out])",
     [P + "test_symmetric_compression_equals_full_sec_5"]),
    ("sci-neighbours-missing", "hifie.py", "_skeletonize",
     "cN = np.nonzero(near | sci)[0]", "cN = np.nonzero(near)[0]",
     [P + "test_sci_coupled_dofs_join_near_field_sec_4_3"]),
    ("no-group-split", "hifie.py", "_skeletonize",
     "groups = sci_groups(M[np.ix_(cN, cbox)]) if second_kind else [np.arange(n)]",
     "groups = [np.arange(n)]",
     [P + "test_sci_groups_lemma_4_2_and_half_edges"]),
    ("top-block-without-sci", "hifie.py", "factor",
     "top_A = op.entries(top, top) + S[np.ix_(top, top)]", "top_A = op.entries(top, top)",
     [P + "test_accuracy_bounds_2d"]),
    ("solve-sweep-sign", "hifie.py", "solve",
     "            x[bf.sk] -= bf.X @ x[bf.rd]\n", "            x[bf.sk] += bf.X @ x[bf.rd]\n",
     [P + "test_sweeps_match_product_formula_eq_4_1"]),
    ("depth-off-by-one", "hifie.py", "num_levels",
     "if np.bincount(flat).max() <= occupancy:", "if np.bincount(flat).max() < occupancy:",
     [PT + "test_depth_is_smallest_with_occupancy_met"]),
    ("edge-range-from-zero", "hifie.py", "centers",
     "ranges = [range(1, s) if t == _I else range(0, s) for t in fam]",
     "ranges = [range(0, s) if t == _I else range(0, s) for t in fam]",
     [PT + "test_2d_edge_centres_are_interior_cell_sides"]),
    ("refine-residual-sign", "krylov.py", "refine",
     "r = f - matvec(u)", "r = matvec(u) - f",
     [PT + "test_refine_contracts_by_norm_of_E"]),
    ("refine-count-off-by-one", "krylov.py", "refine",
     "return u, it, hist", "return u, it + 1, hist",
     [PT + "test_refine_contracts_by_norm_of_E"]),
    ("ldl-no-pivoting", "hifie.py", "ldl_diag_pivot",
     "p = j + int(np.argmax(diag))", "p = j",
     [P + "test_ldl_diag_pivot_reconstructs_and_pivots_on_largest_diagonal"]),
    ("proxy-out-weight-b", "kernels.py", "Operator.proxy_out",
     "(self.w[cols] * self.c[cols])[None, :]", "(self.w[cols] * self.b[cols])[None, :]",
     [P + "test_proxy_rows_span_far_field_lemma_3_3"]),
    ("matvec-ignores-transpose", "kernels.py", "Operator.matvec",
     "Y[rows] = self.entries(idx, rows).T @ X", "Y[rows] = self.entries(rows, idx) @ X",
     [P + "test_direct_sum_rows_match_full"]),
    ("norm2-returns-gram-norm", "idqr.py", "norm2_estimate",
     "return float(np.linalg.norm(Y @ v))", "return float(np.linalg.norm(Y.T @ (Y @ v)))",
     [P + "test_norm2_estimate"]),
    ("apply-transpose-sweep-sign", "hifie.py", "HIFFactor.apply_transpose",
     "x[bf.sk] += bf.Y.T @ x[bf.rd]", "x[bf.sk] -= bf.Y.T @ x[bf.rd]",
     [P + "test_sweeps_match_product_formula_eq_4_1"]),
    ("solve-transpose-top-untransposed", "hifie.py", "HIFFactor.solve_transpose",
     "x[self.top] = lu_solve(self.top_lu, x[self.top], trans=1)", "x[self.top] = lu_solve(self.top_lu, x[self.top])",
     [P + "test_sweeps_match_product_formula_eq_4_1"]),
    ("symmetry-test-ignores-b-c", "hifie.py", "is_symmetric",
     "return bool(np.array_equal(op.b, op.c) and np.all(op.w == op.w[0]))",
     "return bool(np.all(op.w == op.w[0]))",
     [P + "test_symmetry_test_matches_dense_transpose"]),
    ("3d-face-family", "hifie.py", None,
     "(3, \"face\"): [(_I, _H, _H), (_H, _I, _H), (_H, _H, _I)]",
     "(3, \"face\"): [(_I, _H, _H), (_H, _I, _H), (_H, _I, _I)]",
     [PT + "test_3d_face_and_edge_centres_are_interior"]),
    ("root-box-without-cells", "hifie.py", "root_box",
     "lo = (points - 0.5 * side[:, None]).min(axis=0)", "lo = points.min(axis=0)",
     [PT + "test_depth_is_smallest_with_occupancy_met"]),
    ("ldl-never-refuses", "hifie.py", "ldl_diag_pivot",
     "abs(Bw[p, p]) < LDL_ALPHA * colmax", "abs(Bw[p, p]) < 0.0 * colmax",
     [P + "test_ldl_diag_pivot_refuses_weak_pivots"]),
    ("gmres-mgs-sign", "krylov.py", "gmres",
     "wv = wv - H[i, j] * V[:, i]", "wv = wv + H[i, j] * V[:, i]",
     [P + "test_gmres_lemma_5_1_iteration_bound"]),
    ("gmres-unpreconditioned", "krylov.py", "gmres",
     "Z[:, j] = M(V[:, j])", "Z[:, j] = V[:, j]",
     [P + "test_gmres_exact_preconditioner_one_step"]),
    ("power-norm-without-sqrt", "krylov.py", "power_norm",
     "new = np.sqrt(nw)", "new = nw",
     [P + "test_error_estimates_match_dense_two_norms"]),
    ("power-norm-E-E-instead-of-Et-E", "krylov.py", "power_norm",
     "w = apply_op_t(apply_op(v))", "w = apply_op(apply_op(v))",
     [P + "test_error_estimates_match_dense_two_norms"]),
    ("self-term-3d-sign", "kernels.py", "self_integral",
     "(3.0 * math.log(2.0 + math.sqrt(3.0)) - 0.5 * math.pi)", "(3.0 * math.log(2.0 + math.sqrt(3.0)) + 0.5 * math.pi)",
     [P + "test_self_cell_3d_matches_quadrature"]),
    ("ldl-schur-divides-by-D", "hifie.py", "_skeletonize",
     "delta = -(X * Dg[None, :]) @ X.T", "delta = -(X / Dg[None, :]) @ X.T",
     [P + "test_ldl_factor_equals_lu_factor"]),
    ("apply-top-block-transposed", "hifie.py", "HIFFactor.apply",
     "x[self.top] = self.top_A @ x[self.top]", "x[self.top] = self.top_A.T @ x[self.top]",
     [P + "test_sweeps_match_product_formula_eq_4_1"]),
    ("gmres-givens-sign", "krylov.py", "gmres",
     "g[j + 1] = -sn[j] * g[j]", "g[j + 1] = sn[j] * g[j]",
     [P + "test_gmres_lemma_5_1_iteration_bound"]),
    ("helmholtz-self-term-sign", "helmholtz.py", "self_integral_helmholtz",
     "re = part(lambda r: -0.25 * ss.y0(k * r))", "re = part(lambda r: 0.25 * ss.y0(k * r))",
     [PH + "test_self_integral_small_k_limit"]),
    ("helmholtz-block-convention", "helmholtz.py", "EmbeddedOperator.kernel_entries",
     "return np.where(ra == cb, Z.real, np.where(ra == 1, Z.imag, -Z.imag))",
     "return np.where(ra == cb, Z.real, np.where(ra == 1, -Z.imag, Z.imag))",
     [PH + "test_embedded_operator_entries_and_dense_solve"]),
    ("helmholtz-proxy-in-untransposed", "helmholtz.py", "EmbeddedOperator.proxy_in",
     "out[0::2] = np.where(cb == 0, Z.real, Z.imag)\n        out[1::2] = np.where(cb == 0, -Z.imag, Z.real)",
     "out[0::2] = np.where(cb == 0, Z.real, -Z.imag)\n        out[1::2] = np.where(cb == 0, Z.imag, Z.real)",
     [PH + "test_embedded_proxy_blocks_are_operator_blocks"]),
]


def _plant(src, func, old, new):
    """Replace ``old`` by ``new`` exactly once, inside the body of ``func``
    (the def line through the last line indented deeper than it)."""
    if func is None:
        start, end = 0, len(src)
    else:
        lines = src.splitlines(keepends=True)
        cls, _, name = func.rpartition(".")
        lo, hi = 0, len(lines)
        if cls:                                        # a method: search inside its class only
            ch = [i for i, ln in enumerate(lines) if ln.startswith(f"class {cls}(") or ln.startswith(f"class {cls}:")]
            assert len(ch) == 1, f"class {cls} is defined {len(ch)} times"
            lo = ch[0] + 1
            hi = next((i for i in range(lo, len(lines)) if lines[i].strip() and not lines[i][0].isspace()), len(lines))
        heads = [i for i in range(lo, hi) if lines[i].lstrip().startswith(f"def {name}(")]
        assert len(heads) == 1, f"{func} is defined {len(heads)} times"
        h = heads[0]
        indent = len(lines[h]) - len(lines[h].lstrip())
        e = h + 1
        while e < len(lines) and (not lines[e].strip() or len(lines[e]) - len(lines[e].lstrip()) > indent):
            e += 1
        start, end = sum(map(len, lines[:h])), sum(map(len, lines[:e]))
    body = src[start:end]
    assert body.count(old) == 1, f"planted text found {body.count(old)} times in {func}"
    return src[:start] + body.replace(old, new) + src[end:]


PIN_FILES = ("conftest.py", "test_oracle_pins.py", "test_oracle_pins_tree.py", "test_oracle_pins_helmholtz.py")


def _run_case(base, planted, pins):
    """Copy the pins, the input generators and the oracle (with ``planted``:
    (file, function, old, new), or None) under ``base`` and run ``pins``
    there in a fresh interpreter; returns (exit code, output tail)."""
    ign = shutil.ignore_patterns("__pycache__", "*.pyc")
    os.makedirs(base / "tests")
    for f in PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), base / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), base / "tests" / "golden", ignore=ign)
    shutil.copytree(os.path.join(ROOT, "hif_inputs"), base / "hif_inputs", ignore=ign)
    shutil.copytree(os.path.join(ROOT, "oracle"), base / "oracle", ignore=ign)
    if planted is not None:
        fname, func, old, new = planted
        path = base / "oracle" / fname
        path.write_text(_plant(path.read_text(), func, old, new))
    # one BLAS thread per run: the runs themselves go side by side
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *(["-x"] if planted is not None else []), *pins],
                       cwd=base, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, "\n".join((r.stdout + r.stderr).splitlines()[-8:])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    # every case in its own scratch tree, several at a time
    from concurrent.futures import ThreadPoolExecutor
    root = tmp_path_factory.mktemp("mutants")
    jobs = {m[0]: (m[1:5], m[5]) for m in MUTATIONS}
    allpins = sorted({p for m in MUTATIONS for p in m[5]})
    for c in range(6):                                   # the unplanted copy, in six chunks
        jobs[f"unplanted {c}"] = (None, allpins[c::6])
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {k: ex.submit(_run_case, root / f"case{i}", planted, pins)
                for i, (k, (planted, pins)) in enumerate(jobs.items())}
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(outcomes, case):
    rc, tail = outcomes[case[0]]
    assert rc == 1, f"planted mistake not caught (exit {rc}):\n{tail}"


def test_unplanted_copy_passes_the_same_pins(outcomes):
    # the copies themselves are sound: with nothing planted every pin above passes
    bad = {k: v for k, v in outcomes.items() if k.startswith("unplanted ") and v[0] != 0}
    assert not bad, bad
