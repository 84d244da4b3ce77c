"""The oracle's pins catch plausible mistakes (no GPU needed).

Each case copies the oracle's source, plants one mistake of the kind a reader of the paper could make,
builds that variant, and runs the pins of test_oracle.py against it: at least one pin must fail.
"""
import ctypes
import importlib.util
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bsm_oracle.cpp")

MUTANTS = {
    "Eq. 3 strictness": ("gray[(size_t)py * w + px] > gray[(size_t)qy * w + qx]",
                         "gray[(size_t)py * w + px] >= gray[(size_t)qy * w + qx]"),
    "Eq. 3 operand order": ("gray[(size_t)py * w + px] > gray[(size_t)qy * w + qx]",
                            "gray[(size_t)qy * w + qx] > gray[(size_t)py * w + px]"),
    "Eq. 8 precedence": ("(b[j] ^ o[j]) & m[j]", "b[j] ^ (o[j] & m[j])"),
    "Eq. 8 mask of the other view": ("const uint32_t *m = Phiref + ((size_t)y * w + x) * nw;",
                                     "const uint32_t *m = Phiref + ((size_t)y * w + xd) * nw;"),
    "match direction": ("const int xd = dir == 0 ? x - d : x + d;", "const int xd = dir == 0 ? x + d : x - d;"),
    "out-of-image cost": ("if (xd < 0 || xd >= w) return (uint32_t)(32 * nw);", "if (xd < 0 || xd >= w) return 0u;"),
    "Eq. 5 max": ("wgt[i] = std::max(sp, sq);", "wgt[i] = std::min(sp, sq);"),
    "Eq. 5 one term": ("wgt[i] = std::max(sp, sq);", "wgt[i] = sp;"),
    "T rank off by one": ("const int T = sorted[k - 1];", "const int T = sorted[k < n ? k : n - 1];"),
    "Eq. 6 strict": ("if (wgt[i] <= T) m[i / 32]", "if (wgt[i] < T) m[i / 32]"),
    "bit order": ("b[i / 32] |= 1u << (i % 32);", "b[i / 32] |= 1u << (31 - i % 32);"),
    "CIELAB L offset": ("out[0] = (int)std::lround(116.0 * fy - 16.0);", "out[0] = (int)std::lround(116.0 * fy);"),
    "CIELAB b sign": ("out[2] = (int)std::lround(200.0 * (fy - fz));", "out[2] = (int)std::lround(200.0 * (fz - fy));"),
    "sRGB curve": ("return std::pow((c + 0.055) / 1.055, 2.4);", "return std::pow(c, 2.2);"),
    "intensity weights": ("return (77 * px[0] + 150 * px[1] + 29 * px[2] + 128) >> 8;",
                          "return (85 * px[0] + 85 * px[1] + 86 * px[2] + 128) >> 8;"),
    "window short by one": ("for (int dy = -r; dy <= r; ++dy)", "for (int dy = -r; dy < r; ++dy)"),
    "Eq. 1 largest d on ties": ("        if (a < best) {", "        if (a <= best) {"),
    "LR tolerance strict": ("ok = std::abs(d - dR[(size_t)y * w + xr]) <= tol;",
                            "ok = std::abs(d - dR[(size_t)y * w + xr]) < tol;"),
    "LR partner": ("const int xr = x - d;\n      int ok = 0;", "const int xr = x + d;\n      int ok = 0;"),
    "Eq. 10 no distance term": ("const uint32_t v = (uint32_t)(((uint64_t)Ec[c] * Es[e2]) >> 15);",
                                "const uint32_t v = Ec[c];"),
    "Eq. 10 lambda_c": ("Ec[c] = (uint32_t)std::lround(32768.0 * std::exp(-(double)c / lambda_c));",
                        "Ec[c] = (uint32_t)std::lround(32768.0 * std::exp(-(double)c / lambda_e));"),
    "Eq. 9 largest d on ties": ("        if (W[d] > best) {", "        if (W[d] >= best && W[d] > 0) {"),
    "both-mask ablation at x": ("const uint32_t *mo = Phioth + ((size_t)y * w + xd) * nw;",
                                "const uint32_t *mo = Phioth + ((size_t)y * w + x) * nw;"),
    "SGM without the d-1 neighbour": ("if (d > 0) best = std::min(best, prev[d - 1] + P1);", "if (d > 0) best = best;"),
    "SGM without normalisation": ("L[p * dmax + d] = C[p * dmax + d] + best - m;", "L[p * dmax + d] = C[p * dmax + d] + best;"),
    "SGM P2 for P1": ("int64_t best = std::min(prev[d], m + P2);", "int64_t best = std::min(prev[d], m + P1);"),
    "SGM largest d on ties": ("if (sum[p * dmax + d] < sum[p * dmax + arg]) arg = d;",
                              "if (sum[p * dmax + d] <= sum[p * dmax + arg]) arg = d;"),
    "SGM direction reversed": ("const int px = x - dx, py = y - dy;", "const int px = x + dx, py = y + dy;"),
    "fallback max": ("if (left >= 0 && right >= 0) arg = std::min(left, right);",
                     "if (left >= 0 && right >= 0) arg = std::max(left, right);"),
}


def load_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name!r} not found"
    mutated = src.replace(old, new)
    cpp = tmp_path / "variant.cpp"
    so = tmp_path / "variant.so"
    cpp.write_text(mutated)
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(cpp)],
                   check=True)
    spec = importlib.util.spec_from_file_location(f"oracle.variant_{abs(hash(name))}",
                                                  os.path.join(ROOT, "oracle", "oracle.py"),
                                                  submodule_search_locations=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    spec.loader.exec_module(mod)
    mod._lib = mod.bind(ctypes.CDLL(str(so)))
    return mod


def run_pins(variant):
    import test_oracle as pins

    failed = []
    for name in sorted(dir(pins)):
        fn = getattr(pins, name)
        if not name.startswith("test_") or not callable(fn):
            continue
        calls = [dict(shift=s) for s in (0, 3, 7)] if name == "test_constant_shift_recovered" else [{}]
        for kw in calls:
            try:
                fn(variant, **kw)
            except AssertionError:
                failed.append(name)
            except Exception as e:  # a crash or a rejected argument also exposes the mistake
                failed.append(f"{name}: {type(e).__name__}")
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, name):
    old, new = MUTANTS[name]
    variant = load_variant(tmp_path, name, old, new)
    failed = run_pins(variant)
    assert failed, f"no pin caught the planted mistake {name!r}"
