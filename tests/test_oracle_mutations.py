"""The pins have teeth: plausible mistakes planted in a copy of the oracle must fail them.

Each mutant is oracle.c with one textual change (a dropped term, a wrong index,
a transposed operand, a wrong weight), compiled to a temporary library and
swapped in for the duration of the check.  Everything runs on the CPU.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (function whose body is edited, old text, new text, pin that must fail)
MUTANTS = {
    "enum_identity_only": ("mttkrp_enum_range", "} while (next_perm(c, order));", "} while (0);",
                           lambda: pins.test_mttkrp_vs_dense_bruteforce(3, 6, 0)),
    "enum_dropped_factor": ("mttkrp_enum_range", "for (int q = 1; q < order; ++q)", "for (int q = 2; q < order; ++q)",
                            lambda: pins.test_mttkrp_vs_dense_bruteforce(4, 5, 0)),
    "runs_wrong_weight": ("orc_mttkrp_runs", "int64_t den = fact(m[t] - 1);", "int64_t den = fact(m[t]);",
                          lambda: pins.test_paper_normalized_update_counts("runs")),
    "runs_wrong_exponent": ("orc_mttkrp_runs", "int ex = m[s] - (s == t ? 1 : 0);", "int ex = m[s];",
                            lambda: pins.test_mttkrp_vs_dense_bruteforce(3, 6, 1)),
    "ssymv_transposed": ("orc_ssymv_enum", "double t = a * x[c[1]];", "double t = a * x[c[0]];",
                         lambda: pins.test_ssymv_syprd_vs_dense(0)),
    "syprd_no_mirror": ("orc_syprd_enum", "} while (next_perm(c, 2));", "} while (0);",
                        lambda: pins.test_paper_ssymv_syprd_assignments()),
    "canon_unsorted_tuple": ("orc_canonicalize", "sort_tuple(r[e].c, order);", "",
                             lambda: pins.test_canonicalize_properties()),
    "cpfit_sign": ("orc_cpfit", "*res = xx - 2.0 * xm + mm;", "*res = xx + 2.0 * xm + mm;",
                   lambda: pins.test_cpfit_vs_dense(3, 5)),
    "cpals_wrong_power": ("orc_cp_als_step", "for (int q = 0; q < order - 1; ++q) h *= g;",
                          "for (int q = 0; q < order; ++q) h *= g;",
                          lambda: pins.test_cp_als_step_vs_dense(3, 6, 2)),
    "cpals_transposed_solve": ("orc_cp_als_step", "t -= H[k * R + r] * B_new[i * R + k];",
                               "t -= H[r * R + k] * B_new[i * R + k];",
                               lambda: pins.test_cp_als_step_vs_dense(4, 5, 3)),
    "ttm_identity_only": ("orc_ttm_enum", "} while (next_perm(c, order));", "} while (0);",
                          lambda: pins.test_ttm_vs_dense_bruteforce(3, 6, 1)),
    "ttm_wrong_factor_row": ("orc_ttm_enum", "double t = v * B[(int64_t)c[0] * R + r];",
                             "double t = v * B[(int64_t)c[1] * R + r];",
                             lambda: pins.test_paper_ttm_listing_assignments()),
    "pperm_last_part_only": ("next_part_perm", "for (int p = nparts - 1; p >= 0; --p) {",
                             "for (int p = nparts - 1; p >= nparts - 1; --p) {",
                             lambda: pins.test_pmttkrp_vs_dense_bruteforce((2, 2), (4, 3))),
    "pcanon_sort_whole_tuple": ("orc_pcanonicalize", "sort_within_parts(r[e].c, nparts, part);",
                                "sort_tuple(r[e].c, order);", lambda: pins.test_pcanonicalize_properties()),
    "pmttkrp_drops_leading_factors": ("orc_pmttkrp_enum", "if (q != f) t *= fq[q]", "if (q > f) t *= fq[q]",
                                      lambda: pins.test_pmttkrp_vs_dense_bruteforce((1, 2), (4, 5))),
    "pttm_identity_only": ("orc_pttm_enum", "} while (next_part_perm(c, order, nparts, part));", "} while (0);",
                           lambda: pins.test_pttm_vs_dense_bruteforce((1, 2), (4, 5))),
    "pttm_wrong_factor_row": ("orc_pttm_enum", "v * B[(int64_t)c[0] * R + r]", "v * B[(int64_t)c[1] * R + r]",
                              lambda: pins.test_pttm_contracted_again_is_pmttkrp((3,), (5,))),
    "counts_wrong_fibers": ("orc_counts", "if (e == 0 || c[0] != prev[0]) *root_fibers += 1;",
                            "*root_fibers += 1;", lambda: pins.test_counts_closed_forms(3)),
}


def build_mutant(tmp_path, func, old, new):
    src = open(SRC).read()
    start = src.index(func + "(")
    body_at = src.index(old, start)
    mut = src[:body_at] + new + src[body_at + len(old):]
    c = tmp_path / "mut.c"
    c.write_text(mut)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o",
                           str(so), str(c), "-lm"])
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    func, old, new, pin = MUTANTS[name]
    so = build_mutant(tmp_path, func, old, new)
    real = oracle.lib()
    import ctypes
    mut = ctypes.CDLL(so)
    # copy the argument/return types of the real bindings onto the mutant
    for attr in dir(real):
        if attr.startswith("orc_"):
            f, g = getattr(real, attr), getattr(mut, attr)
            g.argtypes, g.restype = f.argtypes, f.restype
    monkeypatch.setattr(oracle, "_lib", mut)
    with pytest.raises((AssertionError, oracle.OracleError)):
        pin()
