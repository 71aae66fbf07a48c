"""Planted mistakes in the CPU oracle: every one is caught by at least one pin.

Each case below is a copy of oracle/npf_oracle.c with one plausible mistake (a dropped 1/N!, a
flipped or missing term of the resonance denominator, a transposed eigenvector matrix, a
conjugated quotient, a wrong Khatri-Rao orientation, a lost minus sign, an off-by-one rank, a
clamp that is not strict or not real, ...). It is compiled with the oracle's own flags and every
pin of test_oracle_pins runs on it through oracle.substituted_library; the unchanged source,
compiled the same way, passes them all. No mutant reads or writes outside its arrays.
"""
import concurrent.futures
import os

import pytest

import oracle
from tests import test_oracle_pins as pins

# (name, text in npf_oracle.c (exactly once), replacement)
MUTANTS = [
    ("h_fact drops 1/N! (Alg. 2 step 4)",
     "s *= invfact;\n                int p[16];\n                p[0] = p1;",
     "int p[16];\n                p[0] = p1;"),
    ("h_brute drops 1/N! (Eq. 4)", "num *= invfact;\n", ""),
    ("h_slab drops 1/N!",
     "s *= invfact;\n            int p[16];\n            for (int m = 0; m < N - 1; ++m)",
     "int p[16];\n            for (int m = 0; m < N - 1; ++m)"),
    ("denominator adds lambda_i instead of subtracting it", "cd D = -lam[i];", "cd D = lam[i];"),
    ("denominator misses lambda_{p_1}", "for (int m = 0; m < N; ++m) D += lam[p[m]];",
     "for (int m = 1; m < N; ++m) D += lam[p[m]];"),
    ("clamp fires at |D| = eps (not strict)", "if (cabs(D) < eps) D = eps;",
     "if (cabs(D) <= eps) D = eps;"),
    ("clamp keeps the phase of D (not real)", "if (cabs(D) < eps) D = eps;",
     "if (cabs(D) < eps) D = eps * D / cabs(D);"),
    ("divide-off mode divides by 2", "if (mode == 1) return 1.0;", "if (mode == 1) return 2.0;"),
    ("quotient conjugated (|Re d| >= |Im d|)", "im = (b - a * r) / den;", "im = (a * r - b) / den;"),
    ("quotient wrong real part (|Im d| > |Re d|)", "re = (a * r + b) / den;",
     "re = (a * r - b) / den;"),
    ("step 2: Phi transposed", "* U[(int64_t)a1 * n + p1];", "* U[(int64_t)p1 * n + a1];"),
    ("step 3: Phi transposed", "U[(int64_t)am * n + pm];", "U[(int64_t)pm * n + am];"),
    ("step 4: Psi transposed", "s += V[(int64_t)i * n + j] * W[(int64_t)j * nN1 + t];",
     "s += V[(int64_t)j * n + i] * W[(int64_t)j * nN1 + t];"),
    ("Eq. 4 brute force: Phi transposed", "term *= U[(int64_t)a[m] * n + p[m]];",
     "term *= U[(int64_t)p[m] * n + a[m]];"),
    ("Khatri-Rao rows and columns of Psi swapped", "s += v[o * n + pm] * V[(int64_t)pm * n + k];",
     "s += v[o * n + pm] * V[(int64_t)k * n + pm];"),
    ("Khatri-Rao factor of p_1 dropped", "total += v[0] * V[(int64_t)p1 * n + k];",
     "total += v[0];"),
    ("Psi_N without the minus sign of Eq. 7", "acc[(int64_t)i * n + k] -= total;",
     "acc[(int64_t)i * n + k] += total;"),
    ("brute-force Psi_N without the minus sign", "out[(int64_t)i * n + k] = -s;",
     "out[(int64_t)i * n + k] = s;"),
    ("last block of p_1 values skipped", "int hi = lo + p1_block < n ? lo + p1_block : n;",
     "int hi = lo + p1_block < n ? lo + p1_block : n - 1;"),
    ("packed rank skips a value per position", "for (int v = lo; v < s[m]; ++v)",
     "for (int v = lo + 1; v < s[m]; ++v)"),
    ("modal slab: Phi transposed on the prefix", "* U[(int64_t)a1 * n + prefix[0]];",
     "* U[(int64_t)prefix[0] * n + a1];"),
    ("modal slab: last lower index with Psi", "s += W[(int64_t)j * n + aN] * U[(int64_t)aN * n + q];",
     "s += W[(int64_t)j * n + aN] * V[(int64_t)aN * n + q];"),
    ("NPF with Phi transposed", "npf[(int64_t)k * n + i] = U[(int64_t)k * n + i] * t;",
     "npf[(int64_t)k * n + i] = U[(int64_t)i * n + k] * t;"),
    ("NPF without the linear part", "cd t = V[(int64_t)i * n + k];", "cd t = 0.0;"),
]


def _pin_cases():
    """Every (name, function, arguments) of the pins, parametrisations expanded."""
    out = []
    for name in sorted(dir(pins)):
        if not name.startswith("test_"):
            continue
        f = getattr(pins, name)
        combos = [{}]
        for m in getattr(f, "pytestmark", []):
            if m.name != "parametrize":
                continue
            argnames = m.args[0]
            argnames = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
            combos = [{**c, **dict(zip(argnames, v if len(argnames) > 1 else (v,)))}
                      for v in m.args[1] for c in combos]
        out += [(name, f, c) for c in combos]
    return out


def _failing_pins(so):
    """The pin cases that fail (or raise) on the library `so`."""
    failed = []
    with oracle.substituted_library(so):
        for name, f, kw in _pin_cases():
            try:
                f(**kw)
            except pytest.skip.Exception:
                pass
            except Exception:                      # an assertion, or NaN/shape trouble
                failed.append(f"{name}{sorted(kw.items()) if kw else ''}")
    return failed


@pytest.fixture(scope="module")
def compiled(tmp_path_factory):
    """The unchanged source and every mutant, compiled in parallel with the oracle's flags."""
    src = open(oracle._SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = [("unchanged", src)]
    for k, (name, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, (name, src.count(old))
        jobs.append((name, src.replace(old, new)))

    def one(k_job):
        k, (name, text) = k_job
        c = os.path.join(d, f"m{k}.c")
        with open(c, "w") as fh:
            fh.write(text)
        return name, oracle.compile_source(c, os.path.join(d, f"libm{k}.so"))

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(one, enumerate(jobs)))


def test_unchanged_source_passes_every_pin(compiled):
    assert _failing_pins(compiled["unchanged"]) == []


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(compiled, name):
    failed = _failing_pins(compiled[name])
    assert failed, f"no pin catches: {name}"
