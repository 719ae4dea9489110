"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of md_oracle.c (on the CPU), compiles
it, routes the oracle front end to it, and runs every pin in
test_oracle_pins.py: at least one pin must fail.  This is what makes the
pins evidence that the oracle computes the definitions it cites.
"""
import inspect
import os

import pytest

from oracle import oracle as O
import test_oracle_pins as pins

_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "md_oracle.c")

MUTATIONS = {
    "drop_attractive_energy": ("double u = 4.0 * e * (s6 * s6 - s6);\n    double fr", "double u = 4.0 * e * (s6 * s6);\n    double fr"),
    "force_factor_12": ("double fr = 24.0 * e * (2.0 * s6 * s6 - s6) / r2; /*", "double fr = 12.0 * e * (2.0 * s6 * s6 - s6) / r2; /*"),
    "newton3_sign": ("a->f[3 * j + k] -= fr * d[k];", "a->f[3 * j + k] += fr * d[k];"),
    "nonstrict_cutoff_search": ("if (r2 < r2max) fn(ctx, i, j, d, r2);\n            }\n        return;",
                                "if (r2 <= r2max) fn(ctx, i, j, d, r2);\n            }\n        return;"),
    "no_minimum_image": ("return d - L * nearbyint(d / L);", "return d + 0.0 * L;"),
    "virial_index_swap": ("csum_add(&a->vir[3], d[0] * (fr * d[1]));", "csum_add(&a->vir[3], d[0] * (fr * d[2]));"),
    "half_cell_shell": ("for (int ox = -1; ox <= 1; ++ox) {", "for (int ox = 0; ox <= 1; ++ox) {"),
    "full_kick": ("hdtm[s] = (0.5 * dt) / mass[s];", "hdtm[s] = dt / mass[s];"),
    "sigma_not_squared": ("double sr2 = (s * s) / r2;\n    double s6 = sr2 * sr2 * sr2;\n    double u",
                          "double sr2 = s / r2;\n    double s6 = sr2 * sr2 * sr2;\n    double u"),
    "rebuild_threshold_full_skin": ("const double half_skin = 0.5 * skin;", "const double half_skin = skin;"),
    "wrap_image_sign": ("image[3 * i + k] += 1;", "image[3 * i + k] -= 1;"),
    "species_index_transposed": ("int32_t t = si * a->nsp + sj;\n    double rc = a->rc[t];\n    if (!(r2 < rc * rc)) return;\n    double s = a->sig[t];",
                                 "int32_t t = si * a->nsp + si;\n    double rc = a->rc[t];\n    if (!(r2 < rc * rc)) return;\n    double s = a->sig[t];"),
    "grad_gprime_factor": ("(4.0 * s6 - 14.0 * s6 * s6)", "(4.0 * s6 - 12.0 * s6 * s6)"),
    "grad_sigma_factor": ("144.0 * e * (4.0 * s6 * s6 - s6)", "72.0 * e * (4.0 * s6 * s6 - s6)"),
    "grad_w_sign": ("w[k] = a->G[3 * i + k] - a->G[3 * j + k];", "w[k] = a->G[3 * i + k] + a->G[3 * j + k];"),
    "grad_hessian_rank1_factor": ("double h = g * w[k] + 2.0 * gp * wd * d[k];", "double h = g * w[k] + gp * wd * d[k];"),
    "grad_energy_sigma": ("csum_add(&a->esig[u], 24.0 * e * (2.0 * s6 * s6 - s6) / s);",
                          "csum_add(&a->esig[u], 24.0 * e * (s6 * s6 - s6) / s);"),
    "grad_pair_index_unordered": ("int32_t u = si <= sj ? si * a->nsp + sj : sj * a->nsp + si;",
                                  "int32_t u = si * a->nsp + sj;"),
    "tbsma_repulsion_once": ("csum_add(&a->rep, 2.0 * phi);", "csum_add(&a->rep, phi);"),
    "tbsma_density_exponent_q": ("double psi = xi * xi * exp(-2.0 * q * (r / r0 - 1.0));\n    double phi = A * exp(-p * (r / r0 - 1.0));\n    csum_add(&a->rho_acc[i], psi);",
                                 "double psi = xi * xi * exp(-q * (r / r0 - 1.0));\n    double phi = A * exp(-p * (r / r0 - 1.0));\n    csum_add(&a->rho_acc[i], psi);"),
    "tbsma_embedding_own_atom_only": ("(a->inv[i] + a->inv[j])", "(2.0 * a->inv[i])"),
    "tbsma_repulsive_force_factor": ("double fr = (2.0 * p / r0) * phi", "double fr = (p / r0) * phi"),
    "tbsma_band_force_sign": ("- (q / r0) * psi * (a->inv[i] + a->inv[j]);", "+ (q / r0) * psi * (a->inv[i] + a->inv[j]);"),
}


def _pin_tests():
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        if "kind" in inspect.signature(fn).parameters:
            for kind in ("gas", "liquid", "threshold"):
                out.append((f"{name}[{kind}]", lambda fn=fn, kind=kind: fn(kind)))
        else:
            out.append((name, fn))
    return out


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_some_pin_catches(mutation):
    src = open(_SRC).read()
    old, new = MUTATIONS[mutation]
    assert src.count(old) == 1, f"mutation anchor not unique: {mutation}"
    lib = O.build_variant(src.replace(old, new), mutation)
    caught = []
    with O.use_library(lib):
        for name, fn in _pin_tests():
            if name == "test_generators":
                continue
            try:
                fn()
            except (AssertionError, pytest.fail.Exception):
                caught.append(name)
            except pytest.skip.Exception:
                pass
    assert caught, f"no pin caught mutation {mutation}"
