"""Plausible mistakes planted in a copy of the oracle must fail the pins.

Each mutant is the oracle source with one textual change (a dropped term, a
wrong sign, a transposed operand or index); it is compiled to a temporary
library and the pins of ``test_oracle_pins.py`` are run against it.  Every
mutant must fail at least one pin, so that a mistake of that kind in the
oracle itself could not go unnoticed.  The mistakes are planted in the
oracle, on the CPU; nothing here touches the CUDA path.
"""
from __future__ import annotations

import os
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_split as split

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "sve_oracle.c")

# (name, original text, planted text)
MUTANTS = [
    ("sign_u4", "double u4 = R->un - a * (tau4 - R->tau);", "double u4 = R->un + a * (tau4 - R->tau);"),
    ("dropped_du_in_sigma", "double sigma = (du + a * (L->tau + R->tau) - (a - b) * p) / b;",
     "double sigma = (a * (L->tau + R->tau) - (a - b) * p) / b;"),
    ("dropped_KDsigma", "double N = dZ + K * D * sigma;", "double N = dZ;"),
    ("a_for_b_in_lambda2", "double lam2 = u1 - b * tau1;", "double lam2 = u1 - a * tau1;"),
    ("swapped_fluctuations", "if (lk < 0.0) o->Am[c] += lk * jump;", "if (lk > 0.0) o->Am[c] += lk * jump;"),
    ("y_frame_not_rotated_back", "a[0] += o.Ap[0] / dy; a[1] += o.Ap[2] / dy; a[2] += o.Ap[1] / dy;",
     "a[0] += o.Ap[0] / dy; a[1] += o.Ap[1] / dy; a[2] += o.Ap[2] / dy;"),
    ("darcy_friction_power", "C = P->f_dw / (8.0 * h * h);", "C = P->f_dw / (8.0 * h);"),
    ("pressure_factor", "c.Pi = 0.5 * P->g * H * H;", "c.Pi = P->g * H * H;"),
    ("cfl_drops_y", "return P->cfl / (Sx / orc_dx(P) + Sy / orc_dy(P));", "return P->cfl / (Sx / orc_dx(P));"),
    ("inflow_direction", "double inward = (side == 0 || side == 2) ? 1.0 : -1.0;",
     "double inward = (side == 0 || side == 2) ? -1.0 : 1.0;"),
    ("zstar_wrong_index", "double Zs = L->Z + K * (tau2 * tau2 - tau1 * tau1);",
     "double Zs = L->Z + K * (tau2 * tau2 - tau4 * tau4);"),
    ("grass_derivative_power", "second = (m - 1.0) * (un * un) * pm3;", "second = (m - 1.0) * un * pm3;"),
    ("D_uses_a_not_a2", "double D = (R->tau - L->tau) + (R->Pi - L->Pi) / (a * a);",
     "double D = (R->tau - L->tau) + (R->Pi - L->Pi) / a;"),
    ("mpm_derivative_factor", "*dq = 8.0 * 1.5 * sqrt(x);", "*dq = 8.0 * sqrt(x);"),
    ("shields_chain_rule", "double d1 = 2.0 * dqs * alpha * (un * un) / speed;",
     "double d1 = dqs * alpha * (un * un) / speed;"),
    ("flvb_coefficient", "*q = 5.7 * x * sqrt(x);", "*q = 8.0 * x * sqrt(x);"),
    ("ribberink_exponent", "*q = 11.0 * pow(x, 1.65);", "*q = 11.0 * pow(x, 1.5);"),
    ("nielsen_uses_excess", "*q = 12.0 * sqrt(ts) * x;", "*q = 12.0 * sqrt(x) * x;"),
    ("camenen_sign", "double e = exp(-4.5 * tcr / ts);", "double e = exp(4.5 * tcr / ts);"),
    ("tangential_velocity_side", "o->v[3] = R->ut;", "o->v[3] = L->ut;"),
    ("bed_update_sign", "double Zn = X->Z[k] - dt * a[3];", "double Zn = X->Z[k] + dt * a[3];"),
    ("wall_not_mirrored", "out[normal] = -in[normal];", "out[normal] = in[normal];"),
    ("bed_step_bound_dropped", "if (raised) a = sqrt(need);", "(void)need;"),
    ("newton_stops_on_halved_step", "if (!halved && fabs(step) <= P->newton_tol * p)",
     "if (fabs(step) <= P->newton_tol * p)"),
    ("celerity_not_doubled_on_retry", "    a = 2.0 * a;\n", "    a = 1.0 * a;\n"),
    # the splitting scheme (reading R13)
    ("split_exner_downwind", "  if (s > 0.0) return QL;", "  if (s > 0.0) return QR;"),
    ("split_exner_sign", "zn[(size_t)j * nx + i] = z[(size_t)j * nx + i] - d;",
     "zn[(size_t)j * nx + i] = z[(size_t)j * nx + i] + d;"),
    ("split_bed_not_held", "  memcpy(z, zn, sizeof(double) * n); /* the bed held fixed", "  /* the bed held fixed"),
    ("split_dy_for_dx", "double d = dt / dx * (fe - fw);", "double d = dt / dy * (fe - fw);"),
    ("split_old_ghosts", "  orc_fill(P, X, h, hu, hv, z);\n  double dt = *dt_used, dx", "  double dt = *dt_used, dx"),
]

# pins run against each mutant: (callable, args)
PINS = [
    (pins.test_riemann_invariants_and_order, ("grass",)),
    (pins.test_riemann_invariants_and_order, ("mpm",)),
    (pins.test_riemann_rankine_hugoniot, ()),
    (pins.test_riemann_reduces_to_suliciu, ()),
    (pins.test_grass_closure_closed_form, (2.0,)),
    (pins.test_grass_closure_closed_form, (3.0,)),
    (pins.test_mpm_closure_closed_form, ("darcy",)),
    (pins.test_shields_laws_against_mpm, ("darcy",)),
    (pins.test_single_step_50_digit, (1,)),
    (pins.test_single_step_50_digit, (2,)),
    (pins.test_mass_conservation, ("walls2d",)),
    (pins.test_cfl_rule, ()),
    (pins.test_riemann_hard_pairs_reach_a_root, ()),
    (split.test_without_transport_the_bed_is_rigid_and_the_flow_that_of_the_coupled_step, ()),
    (split.test_exner_conserves_the_sediment, (1, ("wall", "wall", "wall", "wall"))),
    (split.test_one_step_by_hand, ()),
    (split.test_uniform_flow_moves_no_bed, ()),
]


def _build_mutant(tmp: str, name: str, old: str, new: str) -> oracle.Oracle:
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/present"
    path = os.path.join(tmp, f"mut_{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.build_oracle(force=True, src=path, out=os.path.join(tmp, f"libmut_{name}.so"))
    return oracle.Oracle(lib)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    pytest.importorskip("mpmath")
    with tempfile.TemporaryDirectory() as tmp:
        mut = _build_mutant(tmp, name, old, new)
        caught = []
        for fn, args in PINS:
            try:
                fn(mut, *args)
            except Exception as e:  # an assertion or an oracle error: the pin fired
                caught.append(f"{fn.__name__}{args}: {type(e).__name__}")
        assert caught, f"planted mistake {name} passed every pin"
