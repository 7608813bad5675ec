"""The oracle's pins catch plausible mistakes (no GPU).

Each mutant below plants one plausible mistake in a copy of ``oracle/``, on the CPU: a dropped term, a
wrong sign, index or operand, a missing factor, or a step taken out of order. The pin suite then runs
against the copy, and at least one pin must fail on every mutant. The unmutated copy must pass the same
suite, so a failure means the mistake was caught and not that the copy is broken. The repository's
``oracle/`` itself is never modified. The mutants are grouped under the section or equation whose
statement they break.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")
PIN_FILES = {
    "pins": "test_oracle_pins.py",
    "rmap": "test_oracle_rmap_pins.py",
    "coarse": "test_oracle_coarse_pins.py",
    "adv": "test_oracle_adv_pins.py",
    "table1": "test_oracle_table1.py",
    "surrogate": "test_surrogate_oracle.py",
}

C = "fdirw_oracle.c"
PY = "__init__.py"
SU = "surrogate.py"

# (name, file, old text, new text, which match to replace (None: every match), pin file to run first)
MUTANTS = [
    # Eq. 1 discretised: the face rule and the neighbour of each face
    ("arithmetic_mean_faces", C, "2.0 * a * b / (a + b) : 0.0;", "0.5 * (a + b) : 0.0;", None, "pins"),
    ("y_face_reads_x_neighbour", C, "b = D[i + nx];", "b = D[i + 1];", 0, "pins"),
    ("max_face_sum_drops_lower_x", C, "if (x > 0) s += gx[i - 1];\n", "", 0, "pins"),
    ("max_face_sum_takes_minimum", C, "if (s > best) best = s;", "if (s < best) best = s;", 0, "pins"),
    # Sec. 3.1 march: the flux-form substep
    ("substep_sign_of_lower_x_flux", C, "acc += gx[gi - 1] * (u[li - 1] - ui);",
     "acc += gx[gi - 1] * (ui - u[li - 1]);", 0, "pins"),
    ("substep_lower_y_face_index", C, "if (j > 0)      acc += gy[gi - nx] * (u[li - bx] - ui);",
     "if (j > 0)      acc += gy[gi - 1] * (u[li - bx] - ui);", 0, "pins"),
    ("substep_upper_y_neighbour", C, "if (j + 1 < by) acc += gy[gi] * (u[li + bx] - ui);",
     "if (j + 1 < by) acc += gy[gi] * (u[li + 1] - ui);", 0, "pins"),
    ("substep_drops_upper_z_face", C,
     "                if (l + 1 < bz) acc += gz[gi] * (u[li + (int64_t)bx * by] - ui);\n", "", 0, "pins"),
    ("substep_without_lam", C, "un[li] = ui + lam * acc;", "un[li] = ui + acc;", 0, "pins"),
    # Sec. 3.1 window and offset layout
    ("window_short_on_plus_x", C, "x1 = sx + R > nx - 1 ? nx - 1 : sx + R;",
     "x1 = sx + R - 1 > nx - 1 ? nx - 1 : sx + R - 1;", 0, "pins"),
    ("kernel_offsets_x_z_transposed", C,
     "k_out[(ox + R) + (int64_t)W1 * ((oy + R) + (int64_t)W1 * (oz + R))] =",
     "k_out[(oz + R) + (int64_t)W1 * ((oy + R) + (int64_t)W1 * (ox + R))] =", 0, "pins"),
    ("march_one_substep_short", C, "    for (int k = 0; k < n_sub; k++) {\n        box_step(nx, ny, gx, gy, gz, wx, wy, wz, lam, lama, x0",
     "    for (int k = 1; k < n_sub; k++) {\n        box_step(nx, ny, gx, gy, gz, wx, wy, wz, lam, lama, x0", 0, "pins"),
    # Eq. 8: c' = p c, not p^T c
    ("superpose_transposed", C, "c_out[IDX(x, y, z, nx, ny)] += c_in[s] * k[",
     "c_out[IDX(x, y, z, nx, ny)] += c_in[IDX(x, y, z, nx, ny)] * k[", 0, "pins"),
    ("full_march_one_substep_short", C,
     "    memcpy(u, c_in, sizeof(double) * (size_t)N);\n    for (int k = 0; k < n_sub; k++) {",
     "    memcpy(u, c_in, sizeof(double) * (size_t)N);\n    for (int k = 1; k < n_sub; k++) {", 1, "pins"),
    ("lam_of_divides_by_h", PY, "(dt_macro / n_sub) / (h * h)", "(dt_macro / n_sub) / h", 0, "table1"),
    ("stable_dt_without_h_squared", PY, "else h * h / m", "else h / m", 0, "table1"),
    # per-source radius rule and Eq. 8 with a radius per source
    ("radius_floor_not_ceil", C, "double c = ceil(r);", "double c = floor(r);", 0, "rmap"),
    ("radius_without_factor_two_in_D", C, "double t = 2.0 * D[s];", "double t = D[s];", 0, "rmap"),
    ("radius_times_h", C, "r = r / h;", "r = r * h;", 0, "rmap"),
    ("radius_clamp_min_dropped", C, "Rmap[s] = R < R_min ? R_min : R;", "Rmap[s] = R;", 0, "rmap"),
    ("rmap_scatter_transposed", C, "c_out[IDX(x, y, z, nx, ny)] += c_in[s] * ks[",
     "c_out[IDX(x, y, z, nx, ny)] += c_in[IDX(x, y, z, nx, ny)] * ks[", 0, "rmap"),
    # Eqs. 10-15: coarse mesh
    ("coarse_counts_every_cell", C, "if (liquid[IDX(x, y, z, nx, ny)]) cnt[", "cnt[", 0, "coarse"),
    ("coarse_column_counts_swapped", C, "((double)cnt[J] * S[o]) / (m * (double)cnt[I])",
     "((double)cnt[I] * S[o]) / (m * (double)cnt[J])", 0, "coarse"),
    ("coarse_band_radius_floor", C, "int Rc = (R + B - 1) / B, Wc = 2 * Rc + 1;", "int Rc = R / B, Wc = 2 * Rc + 1;",
     None, "coarse"),
    ("coarse_mapping_sum_not_mean", C, "for (int64_t I = 0; I < NC; I++) if (cnt[I] > 0) C[I] /= (double)cnt[I];",
     "", 0, "coarse"),
    ("coarse_remap_zeroes_solid", C, "? Cn[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] : c_in[i];",
     "? Cn[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] : 0.0;", 0, "coarse"),
    ("mask_keeps_liquid_solid_x_faces", C, "if (!liquid[i] || x + 1 >= nx || !liquid[i + 1]) gx[i] = 0.0;",
     "if (x + 1 >= nx) gx[i] = 0.0;", 0, "coarse"),
    ("coarse_unit_on_solid_cells_too", C, "if (x / B == bx && y / B == by && z / B == bz && liquid[IDX(x, y, z, nx, ny)])",
     "if (x / B == bx && y / B == by && z / B == bz)", 0, "coarse"),
    ("coarse_step_transposed", C, "* ((dy + Rc) + (int64_t)Wc * (dz + Rc))] * C[J];",
     "* ((dy + Rc) + (int64_t)Wc * (dz + Rc))] * C[I];", 0, "coarse"),
    # Eq. 7 and the P_BC c_far term of Eqs. 10 and 14: far field
    ("open_face_without_lam", C, "un[li] += lam * (gb[gi] * (ghost - u[li]));", "un[li] += gb[gi] * (ghost - u[li]);",
     0, "coarse"),
    ("open_faces_counted_once", C, "gb[i] = liquid[i] ? D[i] * (double)faces : 0.0;",
     "gb[i] = liquid[i] && faces ? D[i] : 0.0;", 0, "coarse"),
    ("open_column_divides_by_source_count", C, "open ? S[o] / (double)cnt[I]", "open ? S[o] / (double)cnt[J]", 0,
     "coarse"),
    ("pbc_sum_not_mean", C, "for (int64_t I = 0; I < NC; I++) if (cnt[I] > 0) PBC[I] /= (double)cnt[I];", "", 0,
     "coarse"),
    ("open_face_sign", C, "un[li] += lam * (gb[gi] * (ghost - u[li]));", "un[li] += lam * (gb[gi] * (u[li] - ghost));",
     0, "coarse"),
    ("open_faces_only_low_x", C, "int faces = (x == 0) + (x == nx - 1) +", "int faces = (x == 0) +", 0, "coarse"),
    ("pbc_ghost_at_zero", C, "gb, 1.0, lam, 0, 0, 0, nx, ny, nz, u, un);", "gb, 0.0, lam, 0, 0, 0, nx, ny, nz, u, un);",
     0, "coarse"),
    ("far_field_update_drops_reservoir", C, "*c_far_out = (m_in + V_far * c_far - m_out) / V_far;",
     "*c_far_out = (m_in - m_out) / V_far;", 0, "coarse"),
    ("pbc_term_without_c_far", C, "+= PBC[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] * c_far;",
     "+= PBC[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))];", 0, "coarse"),
    # Eqs. 4-6: interface exchange; Sec. 2: solid diffusion and the order of the coupled step
    ("absorb_liquid_gains", C, "c_out[l] -= m;", "c_out[l] += m;", 0, "coarse"),
    ("absorb_solid_factor_uses_liquid_eq", C, "(cS_eq - c_in[sd]) / cS_eq", "(cS_eq - c_in[sd]) / cL_eq", 0, "coarse"),
    ("absorb_on_same_phase_faces", C, "                    if (liquid[i] == liquid[j]) continue;\n", "", 0, "coarse"),
    ("absorb_skips_z_faces", C, "int has[3] = {x + 1 < nx, y + 1 < ny, z + 1 < nz};", "int has[3] = {x + 1 < nx, y + 1 < ny, 0};",
     0, "coarse"),
    ("absorb_without_dt", C, "double m = k * fL * fS * dt;", "double m = k * fL * fS;", 0, "coarse"),
    ("solid_march_masks_the_liquid", C, "fo_mask_faces(nx, ny, nz, solid, gx, gy, gz);",
     "fo_mask_faces(nx, ny, nz, liquid, gx, gy, gz);", 0, "coarse"),
    ("coupled_step_march_before_exchange", PY,
     "    c1 = absorb(shape, liquid, k, cS_eq, cL_eq, dt, c)\n    c2 = solid_march(shape, D, liquid, lam_s, n_sub_s, c1)\n",
     "    c1 = solid_march(shape, D, liquid, lam_s, n_sub_s, c)\n    c2 = absorb(shape, liquid, k, cS_eq, cL_eq, dt, c1)\n",
     0, "coarse"),
    # Sec. 5: upwind convection
    ("upwind_lower_x_takes_downwind", C, "adv += (w > 0.0 ? w * u[li - 1] : 0.0) - (w < 0.0 ? -w * ui : 0.0);",
     "adv += (w > 0.0 ? w * ui : 0.0) - (w < 0.0 ? -w * ui : 0.0);", 0, "adv"),
    ("upwind_flow_reversed", C, "un[li] = ui + lam * acc + lama * adv;", "un[li] = ui + lam * acc - lama * adv;", 0,
     "adv"),
    ("upwind_lower_y_face_velocity_index", C, "double w = wy[gi - sy];", "double w = wy[gi];", 0, "adv"),
    ("upwind_scaled_by_lam", C, "un[li] = ui + lam * acc + lama * adv;", "un[li] = ui + lam * acc + lam * adv;", 0,
     "adv"),
    ("upwind_upper_x_outflow_sign", C, "adv -= (w > 0.0 ? w * ui : 0.0) - (w < 0.0 ? -w * u[li + 1] : 0.0);",
     "adv += (w > 0.0 ? w * ui : 0.0) - (w < 0.0 ? -w * u[li + 1] : 0.0);", 0, "adv"),
    ("superpose_adv_lam_lama_swapped", PY,
     "fo_superpose_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam), float(lama)",
     "fo_superpose_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lama), float(lam)", 0, "adv"),
    ("liquid_velocity_not_masked", PY,
     "    _load().fo_mask_faces(nx, ny, nz, _pu8(lq), _p(out[0]), _p(out[1]), _p(out[2]))\n    return out\n",
     "    return out\n", 0, "adv"),
    # the learned surrogate of a source's kernel (Sec. 3.1's column of p, predicted)
    ("conv_taps_x_z_transposed", SU, "t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)", "t = (dz + 1) + 3 * (dy + 1) + 9 * (dx + 1)",
     0, "surrogate"),
    ("conv_grad_input_not_flipped", SU, "sl = gp[:, 1 - dz:1 - dz + P, 1 - dy:1 - dy + P, 1 - dx:1 - dx + P]",
     "sl = gp[:, 1 + dz:1 + dz + P, 1 + dy:1 + dy + P, 1 + dx:1 + dx + P]", 0, "surrogate"),
    ("conv_grad_weight_transposed", SU, 'np.einsum("czyx,ozyx->oc", sl, g)', 'np.einsum("czyx,ozyx->co", sl, g)', 0,
     "surrogate"),
    ("backward_ignores_relu", SU, "g = ga * (zs[l - 1] > 0.0)", "g = ga", 0, "surrogate"),
    ("conv_grad_input_drops_edge_tap", SU, "for dx in (-1, 0, 1):", "for dx in (-1, 0):", 1, "surrogate"),
    ("relu_mask_skipped_below_the_head", SU, "g = ga * (zs[l - 1] > 0.0)",
     "g = ga * (zs[l - 1] > 0.0) if l < LAYERS - 1 else ga", 0, "surrogate"),
    ("relu_mask_of_the_layer_above", SU, "g = ga * (zs[l - 1] > 0.0)", "g = ga * (zs[l] > 0.0)", 0, "surrogate"),
    ("loss_gradient_target_sign", SU, "np.where(mask, y - kk, 0.0)", "np.where(mask, y + kk, 0.0)", 0, "surrogate"),
    ("loss_without_predicted_mass", SU, "np.where(mask, y - kk * z + klnk - kk, 0.0)", "np.where(mask, -kk * z + klnk - kk, 0.0)",
     0, "surrogate"),
    ("head_without_exp", SU, "y = np.where(mask, np.exp(zs[-1][0]), 0.0)", "y = np.where(mask, zs[-1][0], 0.0)", 0,
     "surrogate"),
    ("head_not_masked", SU, "y = np.where(mask, np.exp(zs[-1][0]), 0.0)", "y = np.exp(zs[-1][0])", 0, "surrogate"),
    ("bf16_rounds_half_up", SU, "r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "r = (u + 0x8000) & 0xFFFF0000", 0,
     "surrogate"),
    ("feature_log_scale", SU, "np.log10(d) / 8.0 + 1.0", "np.log10(d) / 4.0 + 1.0", 0, "surrogate"),
    ("feature_zero_D_channel", SU, "1.5) if d > 0 else -0.5", "1.5) if d > 0 else 0.0", 0, "surrogate"),
    ("offset_x_channel_along_y", SU, "f[3] = (o / 8.0)[None, None, :]", "f[3] = (o / 8.0)[None, :, None]", 0,
     "surrogate"),
    ("offset_square_scale", SU, "o[None, None, :] ** 2) / 256.0", "o[None, None, :] ** 2) / 192.0", 0, "surrogate"),
]

# The launcher script puts the copy first on the path, checks that the copy is what `import oracle` loads, then
# runs pytest; tests imported afterwards find the copy in sys.modules.
_LAUNCHER = ("import sys; sys.path.insert(0, sys.argv[1]); import oracle; "
           "assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__; "
           "import pytest; sys.exit(pytest.main(sys.argv[2:]))")


def _copy_oracle(dst_root):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst_root, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))


def _plant(dst_root, fname, old, new, which):
    path = os.path.join(dst_root, "oracle", fname)
    with open(path) as f:
        src = f.read()
    n = src.count(old)
    assert n > 0, "mutant text not found"
    if which is None:
        src = src.replace(old, new)
    else:
        assert which < n, "mutant match index out of range"
        at = -1
        for _ in range(which + 1):
            at = src.index(old, at + 1)
        src = src[:at] + new + src[at + len(old):]
    with open(path, "w") as f:
        f.write(src)


def _run_pins(dst_root, first, threads):
    order = [first] + [k for k in PIN_FILES if k != first]
    files = [os.path.join(TESTS, PIN_FILES[k]) for k in order]
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-c", _LAUNCHER, dst_root, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *files]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _workers():
    n = os.cpu_count() or 1
    return max(1, min(8, n)), max(1, n // max(1, min(8, n)))


def test_mutant_texts_are_present():
    """Every planted mistake names text that is in the oracle (so a refactor cannot silently void it)."""
    for name, fname, old, new, which, first in MUTANTS:
        with open(os.path.join(ROOT, "oracle", fname)) as f:
            n = f.read().count(old)
        assert n > (which or 0), name
        assert old != new and first in PIN_FILES, name
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers, threads = _workers()

    def one(m):
        name, fname, old, new, which, first = m
        root = str(tmp_path / name)
        os.makedirs(root)
        _copy_oracle(root)
        if fname is not None:
            _plant(root, fname, old, new, which)
        return name, _run_pins(root, first, threads)

    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, [("control", None, None, None, None, "pins")] + MUTANTS))
    name, r = results[0]
    assert r.returncode == 0, "the unmutated copy fails its pins:\n" + r.stdout[-3000:] + r.stderr[-2000:]
    survivors, crashed = [], []
    for name, r in results[1:]:
        if r.returncode == 0:
            survivors.append(name)
        elif r.returncode != 1:           # 1: tests failed; anything else: a crash or a usage error
            crashed.append((name, r.returncode, (r.stdout + r.stderr)[-800:]))
    assert not crashed, crashed
    assert not survivors, f"mistakes no pin catches: {survivors}"
