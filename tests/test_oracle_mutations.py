"""Each plausible mistake planted in a copy of the oracle breaks a pin.

The copies are compiled from the oracle source with one textual change each
(on the CPU, in a temporary directory); the real oracle is untouched."""
import os

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "ge_oracle.c")

# (name, original text, planted text): each original occurs in the source.
MUTATIONS = [
    ("printed prefactor 1/(3(1+2r))", "double det = 1.0 + 2.0 * r;",
     "double det = 3.0 * (1.0 + 2.0 * r);"),
    ("sign of (r - r^2)", "out[2] = (r - r2) / det;", "out[2] = (r2 - r) / det;"),
    ("(1 - r^2) as (1 + r^2)", "out[1] = (1.0 - r2) / det;", "out[1] = (1.0 + r2) / det;"),
    ("dropped r^2 d term", "t = fma(k[3], d, t);     /* r^2 d       */", ""),
    ("c3 and c4 swapped in (cc)", "t = fma(k[2], c, t);     /* (r-r^2) c   */",
     "t = fma(k[3], c, t);     /* (r-r^2) c   */"),
    ("left neighbour index", "double a = (lo == 0) ? beta_l : u_in[lo - 1];",
     "double a = (lo == 0) ? beta_l : u_in[lo + 1];"),
    ("transposed group operands", "group_update(k, a, b, c, d, &u_out[lo], &u_out[lo + 1]);",
     "group_update(k, a, c, b, d, &u_out[lo], &u_out[lo + 1]);"),
    ("groupings of the two parities swapped", "for (lo = parity; lo + 1 < n; lo += 2) {",
     "for (lo = 1 - parity; lo + 1 < n; lo += 2) {"),
    ("left singleton uses the right wall", "u_out[0] = singleton_update(k, beta_l, u_in[0], far);",
     "u_out[0] = singleton_update(k, beta_r, u_in[0], far);"),
    ("right group neighbour uses the left wall", "double d = (lo + 2 == n) ? beta_r : u_in[lo + 2];",
     "double d = (lo + 2 == n) ? beta_l : u_in[lo + 2];"),
    ("Saul'yev factor 1/(1+2r)", "out[5] = (1.0 - r) / (1.0 + r);",
     "out[5] = (1.0 - r) / (1.0 + 2.0 * r);"),
    ("Saul'yev neighbour weight", "out[4] = r / (1.0 + r);", "out[4] = r / (1.0 + 2.0 * r);"),
    ("right singleton far neighbour", "double far = (n == 1) ? beta_l : u_in[n - 2];",
     "double far = (n == 1) ? beta_l : u_in[n - 1];"),
    ("run starts at the wrong parity", "ge_oracle_step(n, r, beta_l, beta_r, (int)((step0 + s) % 2), src, dst);",
     "ge_oracle_step(n, r, beta_l, beta_r, (int)((step0 + s + 1) % 2), src, dst);"),
    ("no right singleton", "if (((n - parity) % 2) == 1) {", "if (0) {"),
    ("sub-domain roles swapped (width k)", "#define ROLE_A(jj) ((((jj) / k) + parity) % 2 == 0)",
     "#define ROLE_A(jj) ((((jj) / k) + parity) % 2 == 1)"),
    ("A run reads its right neighbour from the wrong side (width k)",
     "u_out[j - 1] = singleton_update(kc, left_new, u_in[j - 1], OLD(j + 1));",
     "u_out[j - 1] = singleton_update(kc, left_new, u_in[j - 1], OLD(j - 1));"),
    ("B run starts from the left wall (width k)", "double right_new = (j == n) ? beta_r : u_out[j];",
     "double right_new = (j == n) ? beta_l : u_out[j];"),
]


def _failing_pins(orc):
    bad = []
    for name, (fn, tol) in P.PINS.items():
        try:
            dev = fn(orc)
        except Exception:  # a mutant may produce NaN or a singular system
            bad.append(name)
            continue
        if not dev <= tol:
            bad.append(name)
    return bad


@pytest.mark.parametrize("label,orig,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, label, orig, planted):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation anchor not unique: {orig!r}"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(orig, planted))
    lib = oracle.load(oracle.compile_oracle(str(src), str(tmp_path / "libmutant.so")))
    bad = _failing_pins(oracle.Oracle(lib))
    assert bad, f"planted mistake '{label}' passed every pin"
