"""Planted mistakes in the CPU oracle: every one is caught by at least one pin.

Each case below is a copy of oracle/npf_oracle.c with one plausible mistake (a dropped 1/N!, a
flipped or missing term of the resonance denominator, a transposed eigenvector matrix, a
conjugated quotient, a wrong Khatri-Rao orientation, a lost minus sign, an off-by-one rank, a
clamp that is not strict or not real, ...). It is compiled with the oracle's own flags and every
pin of test_oracle_pins runs on it through oracle.substituted_library; the unchanged source,
compiled the same way, passes them all. No mutant reads or writes outside its arrays.

The oracle's Python parts (the mode-interaction NPFs of Eqs. 6-9, the mode subset, the swing-model
tensors and the surrogate network) get the same treatment: a copy of the module's source with one
mistake is executed as a fresh module and the pins of that module run against it.
"""
import concurrent.futures
import contextlib
import os
import types

import pytest

import oracle
from tests import test_oracle_interaction, test_oracle_mlp, test_oracle_pins as pins
from tests import test_oracle_subset, test_oracle_swing

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


_ORACLE_DIR = os.path.dirname(oracle._SRC)
# module file -> [(test module, the name under which it holds the oracle module)]
PY_PINS = {
    "__init__.py": [(test_oracle_interaction, "oracle"), (test_oracle_subset, "oracle")],
    "swing.py": [(test_oracle_swing, "swing")],
    "mlp.py": [(test_oracle_mlp, "M")],
}
# (name, module file, text (exactly once), replacement)
PY_MUTANTS = [
    ("Eq. 7 correction of z(0) with the wrong sign", "__init__.py",
     "z = z + delta ** N * psiN(", "z = z - delta ** N * psiN("),
    ("Eq. 7 correction with delta^(N-1)", "__init__.py",
     "z = z + delta ** N * psiN(", "z = z + delta ** (N - 1) * psiN("),
    ("pN1 with phi_ik for phi_ki", "__init__.py", "out[0] = U * z.T", "out[0] = U * z"),
    ("Eqs. 8-9 with zeta in place of the corrected z(0)", "__init__.py",
     "reduce_weights(sysm.tensors[M], n, M, U, V, sysm.lam, z, eps, True, p1_block)",
     "reduce_weights(sysm.tensors[M], n, M, U, V, sysm.lam, delta * V, eps, True, p1_block)"),
    ("weighted contraction without its minus sign", "__init__.py", "    return -acc\n",
     "    return acc\n"),
    ("subset: weights of every mode", "__init__.py", "W[modes] = _c128(V)[modes]",
     "W[:] = _c128(V)"),
    ("subset: rows of every mode", "__init__.py", "out[modes] = -T[modes]", "out[:] = -T"),
    ("swing: no quarter-turn phase per derivative", "swing.py",
     "return G * math.cos(t + N * math.pi / 2) + B * math.sin(t + N * math.pi / 2)",
     "return G * math.cos(t + (N - 1) * math.pi / 2) + B * math.sin(t + (N - 1) * math.pi / 2)"),
    ("swing: sign of the derivatives in delta_k", "swing.py", "(-1) ** b", "(-1) ** a"),
    ("swing: network coefficient without its minus sign", "swing.py",
     "coef = -model.V[j] / (2.0 * model.H[j])", "coef = model.V[j] / (2.0 * model.H[j])"),
    ("swing: reference-bus line dropped", "swing.py",
     "total += _gN(model.Gb[j], model.Bb[j], model.delta[j], N)", "total += 0.0"),
    ("network: relu derivative dropped", "mlp.py", "dz = _q((dz @ W) * (h > 0.0), bf16)",
     "dz = _q(dz @ W, bf16)"),
    ("network: loss derivative without its factor 2", "mlp.py",
     "dz = _q(2.0 * d / (R * wo), bf16)", "dz = _q(d / (R * wo), bf16)"),
    ("network: bias column left out of the gradient", "mlp.py",
     "ha = np.concatenate([h, np.ones((R, 1))], axis=1)",
     "ha = np.concatenate([h, np.zeros((R, 1))], axis=1)"),
    ("bfloat16 rounding by truncation", "mlp.py",
     "r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = (u >> np.uint64(16)) << np.uint64(16)"),
    ("bfloat16 ties rounded away from zero", "mlp.py",
     "r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = ((u + np.uint64(0x8000)) >> np.uint64(16)) << np.uint64(16)"),
]


def _module_from(fname, text):
    path = os.path.join(_ORACLE_DIR, fname)
    mod = types.ModuleType(f"oracle_copy_{fname[:-3]}")
    mod.__file__ = path
    exec(compile(text, path, "exec"), mod.__dict__)
    return mod


@contextlib.contextmanager
def _held_by(targets, mod):
    old = [(t, attr, getattr(t, attr)) for t, attr in targets]
    try:
        for t, attr in targets:
            setattr(t, attr, mod)
        yield
    finally:
        for t, attr, v in old:
            setattr(t, attr, v)


def _failing_py_pins(fname, text):
    mod = _module_from(fname, text)
    failed = []
    with _held_by(PY_PINS[fname], mod):
        for tmod, _ in PY_PINS[fname]:
            for name in sorted(dir(tmod)):
                if name.startswith("test_"):
                    try:
                        getattr(tmod, name)()
                    except pytest.skip.Exception:
                        pass
                    except Exception:
                        failed.append(f"{tmod.__name__}.{name}")
    return failed


@pytest.mark.parametrize("fname", sorted(PY_PINS))
def test_unchanged_python_module_passes_its_pins(fname):
    text = open(os.path.join(_ORACLE_DIR, fname)).read()
    assert _failing_py_pins(fname, text) == []


@pytest.mark.parametrize("name,fname,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_python_mistake_is_caught(name, fname, old, new):
    text = open(os.path.join(_ORACLE_DIR, fname)).read()
    assert text.count(old) == 1, (name, text.count(old))
    assert _failing_py_pins(fname, text.replace(old, new)), f"no pin catches: {name}"
