"""Writes tests/golden/exact_logz.txt from the closed forms in tests/closed_forms.py.

Run from the repository root: python tests/golden/make_exact_logz.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
import closed_forms as cf  # noqa: E402

ROWS = [
    ("free", 2, 1.0, 0.0, lambda: cf.free_field_logz(2, 1.0)),
    ("free", 4, 1.0, 0.0, lambda: cf.free_field_logz(4, 1.0)),
    ("free", 8, 1.0, 0.0, lambda: cf.free_field_logz(8, 1.0)),
    ("free", 16, 1.0, 0.0, lambda: cf.free_field_logz(16, 1.0)),
    ("free", 32, 1.0, 0.0, lambda: cf.free_field_logz(32, 1.0)),
    ("free", 64, 1.0, 0.0, lambda: cf.free_field_logz(64, 1.0)),
    ("one_site", 1, -4.0, 4.0, lambda: cf.one_site_logz(-4.0, 4.0)),
    ("one_site", 1, -4.0, 8.0, lambda: cf.one_site_logz(-4.0, 8.0)),
    ("one_site", 1, -4.0, 16.0, lambda: cf.one_site_logz(-4.0, 16.0)),
    ("torus2", 2, -4.0, 8.0, lambda: cf.two_by_two_logz(-4.0, 8.0)),
    ("torus2", 2, 1.0, 0.0, lambda: cf.two_by_two_logz(1.0, 0.0)),
]

if __name__ == "__main__":
    path = os.path.join(HERE, "exact_logz.txt")
    head = [l for l in open(path) if l.startswith("#")]
    with open(path, "w") as f:
        f.writelines(head)
        for kind, L, m2, lam, fn in ROWS:
            f.write("%s %d %.1f %.1f %.12f\n" % (kind, L, m2, lam, fn()))
