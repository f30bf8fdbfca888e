"""Planted mistakes in the oracle are caught by its pins (CPU).

Each case plants one plausible mistake in the oracle's source (a flipped branch rule, a
dropped Gershgorin radius, traces over halo positions, a transposed assembly, a missing
minimum image, a dropped absolute value, a missing ReLU mask, ...), loads the edited
source as a stand-in module, points the pin modules at it, and runs the pins that cover
that function: at least one must fail.  The unedited oracle passes the same pins (the
rest of the CPU suite), so a failure here means a pin is blind to that mistake.

The mistakes are planted in the oracle only, on the host; nothing here touches the CUDA
path.
"""
import importlib
import sys
import types

import pytest

import synth

PIN_MODULES = ("tests.test_oracle_sp2", "tests.test_oracle_hamiltonian", "tests.test_oracle_graph_partition",
               "tests.test_oracle_mlp", "tests.test_oracle_foe", "tests.test_sequence")


def mutant(modname, edits):
    """The oracle module `modname` with each (old, new) text edit applied once."""
    orig = importlib.import_module(modname)
    with open(orig.__file__) as f:
        src = f.read()
    for old, new in edits:
        assert src.count(old) == 1, (modname, old)
        src = src.replace(old, new)
    mod = types.ModuleType(modname)
    mod.__file__ = orig.__file__
    exec(compile(src, "<%s with a planted mistake>" % modname, "exec"), mod.__dict__)
    return orig, mod


def install(monkeypatch, orig, mod):
    """Point every pin module, and every other oracle module, at the stand-in."""
    for name in PIN_MODULES:
        importlib.import_module(name)
    for name, m in list(sys.modules.items()):
        if m is None or not (name.startswith("oracle.") or name in PIN_MODULES):
            continue
        for attr, val in list(vars(m).items()):
            if val is orig:
                monkeypatch.setattr(m, attr, mod)


def c1(pins):
    """The 8^3 lattice fixture of the SP2 pins, built with whatever H builder is installed."""
    w = synth.lattice(8, seed=0)
    return w, pins.hamiltonian.build_h(w["pos"], w["box"], w["onsite"])


def run_pins(specs):
    """Run pin functions; return (name, exception type) of those that failed.  A pin that
    fails by an exception other than an assertion (the planted mistake made the oracle
    raise, e.g. a sequence that never converges) also counts: the suite goes red."""
    failed = []
    for modname, fname, *args in specs:
        m = sys.modules[modname]
        call = [c1(m) if a == "c1" else a for a in args]
        try:
            getattr(m, fname)(*call)
        except Exception as e:   # noqa: BLE001
            failed.append((fname, type(e).__name__))
    return failed


SP2, HAM, GP, MLP, FOE, SEQ = PIN_MODULES

# (id, oracle module, edits, pins that must catch it)
CASES = [
    ("branch-rule-flipped", "oracle.sp2",
     [("return abs(t2 - n_occ) < abs(2.0 * t1 - t2 - n_occ)", "return abs(t2 - n_occ) > abs(2.0 * t1 - t2 - n_occ)")],
     [(SP2, "test_diagonal_h_gives_step_function"), (SP2, "test_dense_sp2_matches_eigh_and_projector_invariants", "c1")]),
    ("gershgorin-radius-dropped", "oracle.sp2",
     [("return float(np.min(d - off)), float(np.max(d + off))", "return float(np.min(d)), float(np.max(d))")],
     [(SP2, "test_gershgorin_tridiagonal_closed_form"), (SP2, "test_gershgorin_encloses_spectrum", "c1")]),
    ("gershgorin-radius-counts-diagonal", "oracle.sp2",
     [("np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(d)", "np.asarray(abs(H).sum(axis=1)).ravel()")],
     [(SP2, "test_gershgorin_tridiagonal_closed_form")]),
    ("initial-x-reversed", "oracle.sp2",
     [("(e_max * sp.identity(N, format=\"csr\") - H)", "(H - e_min * sp.identity(N, format=\"csr\"))")],
     [(SP2, "test_diagonal_h_gives_step_function"), (SP2, "test_dense_sp2_matches_eigh_and_projector_invariants", "c1")]),
    ("graph-traces-over-halo", "oracle.sp2",
     [("float(np.trace(x[:c, :c])) for x, c in zip(xs, ncore)", "float(np.trace(x)) for x, c in zip(xs, ncore)"),
      ("float(np.trace(s[:c, :c])) for s, c in zip(Ss, ncore)", "float(np.trace(s)) for s, c in zip(Ss, ncore)")],
     [(SP2, "test_graph_traces_are_core_traces", "c1"), (SP2, "test_graph_assembly_support_and_trace", "c1")]),
    ("assembly-transposed", "oracle.sp2",
     [("(np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))\n\n\ndef chebyshev_thresholded",
       "(np.concatenate(vals), (np.concatenate(cols), np.concatenate(rows))), shape=(N, N))\n\n\ndef chebyshev_thresholded")],
     [(SP2, "test_graph_assembly_support_and_trace", "c1")]),
    ("threshold-not-applied", "oracle.sp2",
     [("M = A.multiply(sp.csr_matrix(S, dtype=np.float64))", "M = A")],
     [(SP2, "test_chebyshev_graph_identity", "c1"), (SP2, "test_one_sp2_step_column_identity", "c1")]),
    ("stall-rule-compares-previous-step", "oracle.sp2",
     [("e >= log.e[n - 2]", "e >= log.e[n - 1]")],
     [(SP2, "test_free_mode_stall_rule")]),
    ("chebyshev-c0-not-halved", "oracle.sp2",
     [("    c[0] *= 0.5\n    return c", "    return c")],
     [(FOE, "test_coefficients_reproduce_known_series"), (FOE, "test_foe_complete_graph_equals_fermi_of_eigenvalues")]),
    ("clenshaw-last-step-doubled", "oracle.sp2",
     [("return coeffs[0] * np.eye(m) + x @ b1 - b2", "return coeffs[0] * np.eye(m) + 2.0 * x @ b1 - b2")],
     [(FOE, "test_clenshaw_equals_forward_sum")]),
    ("gap-estimate-inverse-maps-swapped", "oracle.sp2",
     [("        if b:\n            xh, xl = np.sqrt(xh), np.sqrt(xl)", "        if not b:\n            xh, xl = np.sqrt(xh), np.sqrt(xl)")],
     [(SEQ, "test_gap_estimate_exact_for_two_level_system")]),
    ("minimum-image-dropped", "oracle.hamiltonian",
     [("    d = d - box * np.round(d / box)\n    return np.sqrt", "    return np.sqrt")],
     [(HAM, "test_minimum_image_and_cutoff")]),
    ("hopping-decay-length", "oracle.hamiltonian",
     [("DECAY = 0.3 ", "DECAY = 0.33 ")],
     [(HAM, "test_hopping_closed_forms")]),
    ("hopping-sign", "oracle.hamiltonian",
     [("return -1.0 * np.exp(", "return 1.0 * np.exp(")],
     [(HAM, "test_hopping_at_a_is_minus_one")]),
    ("cutoff-too-long", "oracle.hamiltonian",
     [("RCUT = 2.5 ", "RCUT = 2.52 ")],
     [(HAM, "test_minimum_image_and_cutoff"), (HAM, "test_perfect_lattice_shell_count")]),
    ("h2-threshold-without-abs", "oracle.graph",
     [("keep = np.abs(H2.data) >= thresh", "keep = H2.data >= thresh")],
     [(GP, "test_h2_threshold_brute_force")]),
    ("graph-not-symmetrised", "oracle.graph",
     [("A = (A + A.T + sp.identity(", "A = (A + sp.identity(")],
     [(GP, "test_d_threshold_symmetrises")]),
    ("halo-of-first-core-vertex-only", "oracle.partition",
     [("for i in C]))", "for i in C[:1]]))")],
     [(GP, "test_halo_brute_force")]),
    ("halo-before-core", "oracle.partition",
     [("subs.append(np.concatenate([C, halo])", "subs.append(np.concatenate([halo, C])")],
     [(GP, "test_halo_brute_force")]),
    ("cell-id-axes-swapped", "oracle.partition",
     [("return (c[:, 0] * ncell[1] + c[:, 1]) * ncell[2] + c[:, 2]",
       "return (c[:, 2] * ncell[1] + c[:, 1]) * ncell[0] + c[:, 0]")],
     [(GP, "test_cell_ids_closed_form")]),
    ("relu-mask-missing-in-backward", "oracle.mlp",
     [("dh2 = np.outer(dz, w3) * (h2 > 0)", "dh2 = np.outer(dz, w3)")],
     [(MLP, "test_gradient_matches_central_differences")]),
    ("bce-sign", "oracle.mlp",
     [("- y * z +", "+ y * z +")],
     [(MLP, "test_gradient_matches_central_differences"), (MLP, "test_bias_only_network_closed_form")]),
    ("adam-without-bias-correction", "oracle.mlp",
     [("mh = m / (1 - beta1 ** t)", "mh = m")],
     [(MLP, "test_first_adam_step_is_sign_step")]),
    ("weights-not-fp16-rounded", "oracle.mlp",
     [("W1, b1, W2, b2, w3, b3 = unpack(fp16_round(p) if rounded else p, h)\n    a1",
       "W1, b1, W2, b2, w3, b3 = unpack(p, h)\n    a1")],
     [(MLP, "test_rounded_network_uses_fp16_weights")]),
    ("exact-occupies-top-levels", "oracle.exact",
     [("Vo = V[:, :n_occ]", "Vo = V[:, -n_occ:]")],
     [(SP2, "test_dense_sp2_matches_eigh_and_projector_invariants", "c1")]),
    ("thresholded-squares-not-thresholded", "oracle.sp2",
     [("Sq = threshold_to(X @ X, S)", "Sq = (X @ X).tocsr()")],
     [(SP2, "test_thresholded_sp2_one_step_equals_graph_sp2", "c1", 1)]),
    ("thresholded-branch-applied-as-square", "oracle.sp2",
     [("X = Sq if b else (2.0 * X - Sq).tocsr()", "X = Sq")],
     [(SP2, "test_thresholded_sp2_one_step_equals_graph_sp2", "c1", 0)]),
    ("gap-sequence-stops-on-one-level", "oracle.sp2",
     [("while not (1.0 - xh <= tol and xl <= tol):", "while not (1.0 - xh <= tol or xl <= tol):")],
     [(SEQ, "test_gap_sequence_gives_step_function"), (SEQ, "test_gap_sequence_on_lattice_matches_eigh")]),
    ("gap-sequence-two-occupied-levels", "oracle.sp2",
     [("b = choose_square(xh + xl, xh * xh + xl * xl, 1.0)", "b = choose_square(xh + xl, xh * xh + xl * xl, 2.0)")],
     [(SEQ, "test_gap_sequence_gives_step_function")]),
    ("fermi-sign", "oracle.sp2",
     [("return 0.5 * (1.0 - np.tanh(0.5 * z))", "return 0.5 * (1.0 + np.tanh(0.5 * z))")],
     [(FOE, "test_fermi_function_closed_form")]),
    ("foe-half-width-doubled", "oracle.sp2",
     [("xs.append(clenshaw_dense((h - a * np.eye(len(idx))) / b, coeffs))",
       "xs.append(clenshaw_dense((h - a * np.eye(len(idx))) / (2.0 * b), coeffs))")],
     [(FOE, "test_foe_complete_graph_equals_fermi_of_eigenvalues")]),
    ("tree-build-one-sided", "oracle.hamiltonian",
     [("rows = np.concatenate([i, j, np.arange(N)])", "rows = np.concatenate([i, i, np.arange(N)])")],
     [(HAM, "test_tree_build_equals_brute_force", "lattice")]),
    ("eq8-paths-of-length-one", "oracle.graph",
     [("A2 = (A @ A).tocsr()", "A2 = A.tocsr()")],
     [(GP, "test_eq8_and_hk_brute_force")]),
    ("eq8-without-h-pattern", "oracle.graph",
     [("A = (d_threshold(D, tau).astype(np.int64) + pattern(H).astype(np.int64)).tocsr()",
       "A = d_threshold(D, tau).astype(np.int64).tocsr()")],
     [(GP, "test_eq8_and_hk_brute_force")]),
    ("hk-one-power-short", "oracle.graph",
     [("for _ in range(k - 1):", "for _ in range(k - 2):")],
     [(GP, "test_eq8_and_hk_brute_force")]),
    ("h2-rows-without-abs", "oracle.graph",
     [("R = sp.csr_matrix((np.abs(R.data) >= thresh, R.indices, R.indptr), shape=R.shape)",
       "R = sp.csr_matrix((R.data >= thresh, R.indices, R.indptr), shape=R.shape)")],
     [(GP, "test_h2_threshold_rows_equals_full")]),
    ("candidates-without-minimum-image", "oracle.mlp",
     [("        d = d - box * np.round(d / box)\n        r = np.sqrt", "        r = np.sqrt")],
     [(MLP, "test_candidate_pairs_simple_cubic_shells", 1.5, 18)]),
    ("h2-feature-is-h", "oracle.mlp",
     [("h2ij = np.asarray(H[I].multiply(H[J]).sum(axis=1)).ravel()", "h2ij = hij")],
     [(MLP, "test_h2_feature_equals_matrix_square")]),
    ("onsite-feature-not-symmetrised", "oracle.mlp",
     [("f[:, 3] = np.minimum(onsite[I], onsite[J])", "f[:, 3] = onsite[I]")],
     [(MLP, "test_pairs_and_features_symmetric")]),
    ("hopping-feature-scale", "oracle.mlp",
     [("f[:, 0] = -np.log10(np.maximum(np.abs(hij), 1e-12)) / 12.0", "f[:, 0] = -np.log10(np.maximum(np.abs(hij), 1e-12)) / 10.0")],
     [(MLP, "test_pairs_and_features_symmetric")]),
    ("labels-of-signed-d", "oracle.mlp",
     [("return (np.abs(np.asarray(D[I, J]).ravel()) >= tau)", "return (np.asarray(D[I, J]).ravel() >= tau)")],
     [(MLP, "test_labels_threshold_the_magnitude")]),
    ("graph-from-logits-drops-h", "oracle.mlp",
     [("return graph._finish(E + graph.pattern(H))", "return graph._finish(E)")],
     [(MLP, "test_graph_from_logits_limits_and_example")]),
]


@pytest.mark.parametrize("modname,edits,pins", [c[1:] for c in CASES], ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, modname, edits, pins):
    orig, mod = mutant(modname, edits)
    install(monkeypatch, orig, mod)
    failed = run_pins(pins)
    assert failed, "no pin caught the planted mistake"


def test_unplanted_oracle_passes_the_same_pins():
    """Control: every pin call above passes on the real oracle, so a failure under a
    planted mistake is the mistake's doing (not a mis-specified call)."""
    for name in PIN_MODULES:
        importlib.import_module(name)
    specs = sorted({tuple(p) for c in CASES for p in c[3]}, key=repr)
    assert run_pins(specs) == []
