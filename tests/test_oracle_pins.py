"""The CPU oracle against its pins (see tests/oracle_pins.py), and planted
mistakes in a copy of the oracle's source, each of which a pin must catch."""
import os

import pytest

import oracle
from tests import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check()


# (original text, planted mistake) pairs in hist_oracle.c
MUTANTS = [
    ("return 1 + (int32_t)q;", "return (int32_t)q;"),                       # dropped +1
    ("if (x < edges[mid])", "if (x <= edges[mid])"),                        # lower_bound search
    ("if (q >= (double)nbins) return nbins; /* R3 */", ""),                 # no clamp
    ("term[5] = wy * y;", "term[5] = wx * y;"),                             # wrong operand
    ("term[3] = wx * x;", "term[3] = wx;"),                                 # dropped factor
    ("double d = x - xmin;", "double d = xmin - x;"),                       # wrong sign
    ("double q = t / (xmax - xmin);", "double q = t / (xmin - xmax);"),     # transposed operands
    ("stride *= (int64_t)axes[d].nbins + 2;", "stride *= (int64_t)axes[d].nbins + 1;"),
    ("if (!in_range && !stat_overflows) continue;", "if (!in_range && stat_overflows) continue;"),
    ("*c += (*s - t) + v;", "*c += (*s - t) - v;"),                         # broken compensation
    ("term[1] = w * w;", "term[1] = w;"),                                   # dropped square
    ("if (!(x < edges[nbins])) return nbins + 1;", "if (x > edges[nbins]) return nbins + 1;"),
    ("if (b < 1 || b > axes[d].nbins) in_range = 0;", "if (b < 1) in_range = 0;"),
    ("term[9] = wx * z;", "term[9] = wy * z;"),
    ("o->bins_seq[g] += w;", "o->bins_seq[g] += fabs(w);"),
    # the chunk-parallel modes: split, merge, compensation merge, locate
    ("j->i1 = n * (t + 1) / nthreads;", "j->i1 = n * (t + 1) / nthreads - (t + 1 < nthreads);"),
    ("counts[g] += p->counts[g];", "counts[g] = p->counts[g];"),
    ("neumaier_add(&bins_acc_s[g], &bins_acc_c[g], p->bins_acc_c[g]);", ""),
    ("neumaier_add(&stats_acc_s[k], &stats_acc_c[k], p->stats_acc_c[k]);", ""),
    ("bins_seq[g] += p->bins_seq[g];", "bins_seq[g] = p->bins_seq[g];"),
    ("int32_t b = find_bin(&j->axes[d], j->values[(int64_t)d * j->n + i]);",
     "int32_t b = find_bin(&j->axes[d], j->values[(int64_t)d * j->n + i - (i > j->i0)]);"),
]


@pytest.mark.parametrize("old,new", MUTANTS, ids=[f"m{i}" for i in range(len(MUTANTS))])
def test_planted_mistake_is_caught(old, new, tmp_path):
    src = oracle.source_text()
    assert old in src, f"mutation anchor not found: {old!r}"
    mutant = src.replace(old, new)
    so = oracle.compile_variant(mutant, os.path.join(str(tmp_path), "libmutant.so"))
    failures = []
    with oracle.use_library(so):
        for check in P.ALL_CHECKS:
            try:
                check()
            except AssertionError as e:
                failures.append((check.__name__, str(e)[:120]))
                break
    assert failures, f"no pin caught the planted mistake {old!r} -> {new!r}"
