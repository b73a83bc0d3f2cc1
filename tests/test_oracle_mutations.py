"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (a dropped factor, a wrong sign, a
transposed or conjugated operand, an off-by-one index), on the CPU, through
monkeypatch, and runs the pin that must then fail. A pin that still passed
would leave that mistake invisible to every parity test built on the oracle.
"""
import numpy as np
import pytest

import test_oracle_dft as t_dft
import test_oracle_pft as t_pft
import test_oracle_pie as t_pie
import test_oracle_tv as t_tv
from oracle import coeffs, dft, grad, pft, pie, tv
from paper_2408_03532_gb300 import synth


def fails(check, *args):
    with pytest.raises((AssertionError, ValueError, IndexError)):
        check(*args)


# ---------------------------------------------------------------- Algorithm 1 tables
def test_twiddle_table_without_its_phase_factor(monkeypatch):
    orig = coeffs.plan_1d

    def bad(*a, **k):
        P = orig(*a, **k)
        P["W"] = P["W"] * np.exp(1j * np.pi * P["t"] / P["p"])[:, None]  # e^{-i pi t/p} dropped
        return P
    monkeypatch.setattr(coeffs, "plan_1d", bad)
    fails(t_pft.test_1d_error_bound, 64, 32, 16)


def test_abscissae_with_the_wrong_sign(monkeypatch):
    orig = coeffs.plan_1d

    def bad(*a, **k):
        P = orig(*a, **k)
        x = 2.0 * np.arange(P["q"]) / P["q"] - 1.0                        # 2l/q - 1 instead of 1 - 2l/q
        P["B"] = P["w"][None, :] * x[:, None] ** np.arange(P["r"])[None, :]
        return P
    monkeypatch.setattr(coeffs, "plan_1d", bad)
    fails(t_pft.test_1d_error_bound, 64, 32, 16)


# ---------------------------------------------------------------- Algorithm 2 / 5
def test_column_major_reshape(monkeypatch):
    def bad(z, plan):
        p, q, t = plan["p"], plan["q"], plan["t"]
        Chat = np.fft.fft(z.reshape(q, p).T @ plan["B"], axis=0)          # z_{k + p l} instead of z_{q k + l}
        return np.array([np.sum(Chat[tt % p, :] * plan["W"][a, :]) for a, tt in enumerate(t)])
    monkeypatch.setattr(pft, "pft1", bad)
    fails(t_pft.test_1d_error_bound, 64, 32, 16)


def test_residue_off_by_one(monkeypatch):
    def bad(z, plan):
        p, q, t = plan["p"], plan["q"], plan["t"]
        Chat = np.fft.fft(z.reshape(p, q) @ plan["B"], axis=0)
        return np.array([np.sum(Chat[(tt + 1) % p, :] * plan["W"][a, :]) for a, tt in enumerate(t)])
    monkeypatch.setattr(pft, "pft1", bad)
    fails(t_pft.test_1d_error_bound, 64, 32, 16)


def _pft2_frames_variant(stage_b_inverse=False, conj_w=False, swap_tables=False):
    def frames(z, plan1, plan2):
        p1, q1, p2, q2 = plan1["p"], plan1["q"], plan2["p"], plan2["q"]
        B1, B2, W1, W2 = plan1["B"], plan2["B"], plan1["W"], plan2["W"]
        if swap_tables:
            B1, B2, W1, W2 = B2, B1, W2, W1
        if conj_w:
            W1 = W1.conj()
        lead = z.shape[:-2]
        Z = np.moveaxis(z.reshape(*lead, p1, q1, p2, q2), -3, -2)
        C = np.einsum("lj,...abls,sk->...abjk", B1, Z, B2, optimize=True)
        if stage_b_inverse:
            Chat = np.fft.ifft2(C, axes=(-4, -3)) * (p1 * p2)
        else:
            Chat = np.fft.fft2(C, axes=(-4, -3))
        G = Chat[..., np.mod(plan1["t"], p1), :, :, :][..., np.mod(plan2["t"], p2), :, :]
        return np.einsum("...abjk,aj,bk->...ab", G, W1, W2, optimize=True)
    return frames


@pytest.mark.parametrize("kind", ["stage_b_inverse", "conj_w"])
def test_stage_b_sign_and_conjugated_twiddles(monkeypatch, kind):
    monkeypatch.setattr(pft, "_pft2_frames", _pft2_frames_variant(**{kind: True}))
    fails(t_pft.test_2d_error_bound, 64, 64, 32, 32, 16, 16)


def test_tables_of_the_two_axes_swapped(monkeypatch):
    monkeypatch.setattr(pft, "_pft2_frames", _pft2_frames_variant(swap_tables=True))
    fails(t_pft.test_2d_error_bound, 32, 64, 16, 32, 8, 16)


def _pft2_adjoint_variant(conj_w=True, scale=True):
    def frames(y, plan1, plan2):
        p1, q1, r1 = plan1["p"], plan1["q"], plan1["r"]
        p2, q2, r2 = plan2["p"], plan2["q"], plan2["r"]
        B1, B2, W1, W2 = plan1["B"], plan2["B"], plan1["W"], plan2["W"]
        lead = y.shape[:-2]
        G = np.einsum("...ab,aj,bk->...abjk", y, W1.conj() if conj_w else W1, W2.conj(), optimize=True)
        H = np.zeros((*lead, p1, p2, r1, r2), dtype=np.complex128)
        for a, u1 in enumerate(np.mod(plan1["t"], p1)):
            for b, u2 in enumerate(np.mod(plan2["t"], p2)):
                H[..., u1, u2, :, :] += G[..., a, b, :, :]
        E = np.fft.ifft2(H, axes=(-4, -3)) * ((p1 * p2) if scale else 1)
        Z = np.einsum("lj,...abjk,sk->...abls", B1.conj(), E, B2.conj(), optimize=True)
        return np.moveaxis(Z, -2, -3).reshape(*lead, p1 * q1, p2 * q2)
    return frames


@pytest.mark.parametrize("kind", [dict(conj_w=False), dict(scale=False)])
def test_adjoint_without_conjugate_or_scale(monkeypatch, kind):
    monkeypatch.setattr(pft, "_pft2_adjoint_frames", _pft2_adjoint_variant(**kind))
    fails(t_pft.test_adjoint_identity, 64, 64, 32, 32, 16, 16)


# ---------------------------------------------------------------- exact DFT
def test_dft_with_the_wrong_exponent_sign(monkeypatch):
    def bad(n, t):
        k = np.arange(n)
        return np.exp(2j * np.pi * np.mod(np.outer(np.asarray(t, dtype=np.int64), k), n) / n)
    monkeypatch.setattr(dft, "dft_matrix", bad)
    fails(t_dft.test_brute_force_matches_matrix_and_fft_routes, 8, 8, 4, 6)


def test_partial_dft_with_a_conjugate_transposed_factor(monkeypatch):
    def bad(z, M1, M2):
        n1, n2 = z.shape[-2:]
        return dft.dft_matrix(n1, coeffs.freqs(M1)) @ z @ dft.dft_matrix(n2, coeffs.freqs(M2)).conj().T  # F2^H for F2^T
    monkeypatch.setattr(dft, "partial_dft2", bad)
    fails(t_dft.test_brute_force_matches_matrix_and_fft_routes, 8, 8, 4, 6)


# ---------------------------------------------------------------- PIE update (Eq. pie_update, Eq. 3)
def _pie_update_variant(conj_probe=True, normalise=True, residual_sign=1.0):
    def update(obj, probe, pos, d, T, beta, probe_max2):
        n1, n2 = probe.shape
        r, c = int(pos[0]), int(pos[1])
        patch = obj[r:r + n1, c:c + n2]
        Psi = T["fwd"](probe * patch)
        mag = np.abs(Psi)
        phase = np.where(mag > 0.0, Psi / np.where(mag > 0.0, mag, 1.0), 1.0)
        R = Psi - residual_sign * d * phase
        dpsi = T["adj"](R) / ((n1 * n2) if normalise else 1)
        w = np.conj(probe) if conj_probe else probe
        obj[r:r + n1, c:c + n2] = patch - beta * w / probe_max2 * dpsi
        return float(np.sum(np.abs(R) ** 2)) / (n1 * n2)
    return update


def test_update_without_the_conjugate_probe(monkeypatch):
    monkeypatch.setattr(pie, "pie_update", _pie_update_variant(conj_probe=False))
    fails(t_pie.test_batched_equals_sequential_without_overlap)


@pytest.mark.parametrize("kind", [dict(normalise=False), dict(residual_sign=-1.0)])
def test_update_without_normalisation_or_with_the_wrong_residual(monkeypatch, kind):
    monkeypatch.setattr(pie, "pie_update", _pie_update_variant(**kind))
    fails(t_pie.test_full_update_is_the_modulus_projection)


@pytest.mark.parametrize("kind", ["no_division", "modulus_not_squared"])
def test_batched_step_with_a_wrong_illumination(monkeypatch, kind):
    orig = pie.illumination

    def bad(probe, positions, shape):
        if kind == "no_division":
            return np.ones(shape)                                           # the division dropped
        return orig(np.sqrt(np.abs(probe)), positions, shape)               # sum |w| instead of |w|^2
    monkeypatch.setattr(pie, "illumination", bad)
    fails(t_pie.test_batched_step_projects_a_single_exit_wave)


def test_error_metric_with_the_conjugate_phase(monkeypatch):
    def bad(z, truth, mask=None):
        if mask is not None:
            z, truth = z[mask], truth[mask]
        ip = np.vdot(z, truth)
        ph = np.conj(ip) / abs(ip)                                          # aligns the wrong way
        return float(np.linalg.norm(ph * z - truth) / np.linalg.norm(truth))
    monkeypatch.setattr(pie, "nrmse", bad)
    fails(t_pie.test_truth_is_a_fixed_point_and_phase_invariance)


def test_colouring_that_ignores_overlap_in_one_axis(monkeypatch):
    monkeypatch.setattr(pie, "overlaps", lambda a, b, n1, n2: abs(int(a[0]) - int(b[0])) < n1)
    orig = pie.greedy_colouring
    # validity is checked against the true overlap relation
    true_overlaps = lambda a, b, n1, n2: abs(int(a[0]) - int(b[0])) < n1 and abs(int(a[1]) - int(b[1])) < n2

    def check():
        pos = synth.fermat_scan(256, 32, 200)
        col = orig(pos, 32, 32)
        for j in range(len(pos)):
            earlier = {int(col[i]) for i in range(j) if true_overlaps(pos[i], pos[j], 32, 32)}
            assert set(range(col[j])) <= earlier
    fails(check)


# ---------------------------------------------------------------- gradient and TV
def _small_gradient_problem():
    obj = synth.make_object(96)
    probe = synth.make_probe(32)
    pos = synth.raster_scan(4, 4, 16, 8)
    P1, P2 = coeffs.plan_2d(32, 32, 16, 16, 8, 8)
    T = pie.pft_transform(P1, P2)
    d = pie.amplitudes(synth.simulate_intensities(obj, probe, pos), 16)
    return synth.random_init(96), probe, pos, d, T


def _gradient_pin(z, probe, pos, d, T):
    """The pin of the object and probe gradients (FP64 central differences)."""
    _, gz, gw = grad.amplitude_loss_grad(z, probe, pos, d, T)
    rng = np.random.default_rng(0)
    for _ in range(6):
        r, c = 8 + int(rng.integers(80)), 8 + int(rng.integers(80))
        fd = grad.finite_difference(lambda zz: grad.amplitude_loss(zz, probe, pos, d, T), z, (r, c))
        assert abs(fd - gz[r, c]) <= 1e-5 * np.abs(gz).max()
        u, v = int(rng.integers(32)), int(rng.integers(32))
        fd = grad.finite_difference(lambda ww: grad.amplitude_loss(z, ww, pos, d, T), probe, (u, v))
        assert abs(fd - gw[u, v]) <= 1e-5 * np.abs(gw).max()


def test_gradient_pin_passes_on_the_oracle():
    _gradient_pin(*_small_gradient_problem())


@pytest.mark.parametrize("kind", ["factor", "conj"])
def test_gradient_without_its_factor_or_conjugate(monkeypatch, kind):
    orig = grad.amplitude_loss_grad

    def bad(z, probe, positions, d, T):
        loss, gz, gw = orig(z, probe, positions, d, T)
        if kind == "factor":
            return loss, gz / 2.0, gw / 2.0                                 # g_psi = A^H R, the 2 dropped
        return loss, gz.conj(), gw                                          # d/dRe - i d/dIm
    monkeypatch.setattr(grad, "amplitude_loss_grad", bad)
    fails(_gradient_pin, *_small_gradient_problem())


def test_tv_gradient_with_the_wrong_sign(monkeypatch):
    orig = tv.tv_grad
    monkeypatch.setattr(tv, "tv_grad", lambda z, eps: -orig(z, eps))
    fails(t_tv.test_gradient_matches_central_differences)


def test_tv_with_a_backward_difference_adjoint(monkeypatch):
    def bad(u):
        u = np.array(u, copy=True)
        u[:, -1] = 0
        out = np.zeros_like(u)
        out[:, 1:] -= u[:, :-1]                                             # signs of D_x^H swapped
        out[:, :-1] += u[:, :-1]
        return out
    monkeypatch.setattr(tv, "dx_adjoint", bad)
    fails(t_tv.test_difference_adjoints)


def test_tv_step_uphill(monkeypatch):
    monkeypatch.setattr(tv, "tv_step", lambda z, lam, eps: z + lam * tv.tv_grad(z, eps))
    fails(t_tv.test_constant_and_ramp)


# ---------------------------------------------------------------- metrics and the offline phase
def test_error_metric_that_ignores_its_mask(monkeypatch):
    orig = pie.nrmse
    monkeypatch.setattr(pie, "nrmse", lambda z, truth, mask=None: orig(z, truth))
    fails(t_pie.test_error_metrics_closed_forms)


def test_relative_change_against_the_new_iterate(monkeypatch):
    monkeypatch.setattr(pie, "relative_change",
                        lambda new, old: float(np.linalg.norm(new - old) / np.linalg.norm(new)))
    fails(t_pie.test_error_metrics_closed_forms)


def test_one_term_too_many(monkeypatch):
    orig = coeffs.choose_r
    monkeypatch.setattr(coeffs, "choose_r", lambda eps, ratio, r_max=40: orig(eps, ratio, r_max) + 1)
    import test_oracle_coeffs as t_coeffs
    fails(t_coeffs.test_r_matches_paper_value)


def test_taylor_coefficients_instead_of_the_best_approximation(monkeypatch):
    import math
    import test_oracle_coeffs as t_coeffs

    def taylor(xi, r):
        w = np.array([(1j * math.pi) ** j / math.factorial(j) for j in range(r)])
        return w, coeffs.uniform_error(w, xi)
    monkeypatch.setattr(coeffs, "best_approximation", taylor)
    fails(t_coeffs.test_best_error_between_bessel_bounds, 8, 1.0)


# ---------------------------------------------------------------- data, blind PIE, probe gradient
def test_crop_one_frequency_off(monkeypatch):
    def bad(d, M1, M2):
        n1, n2 = d.shape[-2:]
        i1 = np.mod(coeffs.freqs(M1) + 1, n1)                               # t + 1 instead of t
        i2 = np.mod(coeffs.freqs(M2), n2)
        return d[..., i1, :][..., :, i2]
    monkeypatch.setattr(dft, "crop_centre", bad)
    fails(t_dft.test_crop_centre_matches_shifted_crop)


def test_amplitudes_without_the_square_root(monkeypatch):
    monkeypatch.setattr(pie, "amplitudes", lambda I, M=None: np.asarray(I, dtype=np.float64) if M is None
                        else dft.crop_centre(np.asarray(I, dtype=np.float64), M, M))
    fails(t_pie.test_truth_is_a_fixed_point_and_phase_invariance)


@pytest.mark.parametrize("kind", ["conj_probe", "unnormalised"])
def test_blind_probe_step_with_the_wrong_factor(monkeypatch, kind):
    def bad(obj, probe, positions, data, T, beta, gamma, colours, order=None, delta_rel=1e-3):
        n1, n2 = probe.shape
        z = np.array(obj, dtype=np.complex128, copy=True)
        w = np.array(probe, dtype=np.complex128, copy=True)
        cm = pie.colour_major_order(colours, order)
        tot = 0.0
        for c in range(int(colours.max()) + 1):
            members = [j for j in cm if colours[j] == c]
            wmax2 = float(np.max(np.abs(w) ** 2))
            for j in members:
                tot += pie.pie_update(z, w, positions[j], data[j], T, beta, wmax2)
            acc, den = np.zeros_like(w), np.zeros(w.shape)
            for j in members:
                r, cc = positions[j]
                zj = z[r:r + n1, cc:cc + n2]
                R = pie.residual(T["fwd"](w * zj), data[j])
                acc += (np.conj(w) if kind == "conj_probe" else np.conj(zj)) * T["adj"](R) / (n1 * n2)
                den += np.abs(zj) ** 2
            w = w - gamma * acc / ((den + delta_rel * den.max()) if kind == "conj_probe" else 1.0)
        return z, w, tot / len(positions)
    monkeypatch.setattr(pie, "epie_colour_sweep", bad)
    fails(t_pie.test_epie_single_position_probe_step)


def test_probe_gradient_without_the_conjugate_patch(monkeypatch):
    orig = grad.amplitude_loss_grad

    def bad(z, probe, positions, d, T):
        n1, n2 = probe.shape
        loss, gz, _ = orig(z, probe, positions, d, T)
        P = np.stack([z[r:r + n1, c:c + n2] for r, c in positions])
        Psi = T["fwd"](probe[None] * P)
        mag = np.abs(Psi)
        R = Psi - d * np.where(mag > 0.0, Psi / np.where(mag > 0.0, mag, 1.0), 0.0)
        return loss, gz, np.sum(P * 2.0 * T["adj"](R), axis=0)              # Q_j z instead of conj(Q_j z)
    monkeypatch.setattr(grad, "amplitude_loss_grad", bad)
    fails(_gradient_pin, *_small_gradient_problem())


# ---------------------------------------------------------------- Eq. epie_probe_update, sequential
def _bad_epie_sweep(kind):
    def bad(obj, probe, positions, data, T, beta, gamma, order=None):
        n1, n2 = probe.shape
        z = np.array(obj, dtype=np.complex128, copy=True)
        w = np.array(probe, dtype=np.complex128, copy=True)
        order = range(len(positions)) if order is None else order
        acc = np.zeros_like(w)
        tot = 0.0
        for j in order:
            r, c = int(positions[j][0]), int(positions[j][1])
            zold = z[r:r + n1, c:c + n2].copy()
            tot += pie.pie_update(z, w, positions[j], data[j], T, beta, float(np.max(np.abs(w) ** 2)))
            zj = zold if kind == "old_patch" else z[r:r + n1, c:c + n2]
            R = pie.residual(T["fwd"](w * zj), data[j])
            g = (zj if kind == "no_conj" else np.conj(zj)) * (T["adj"](R) / (n1 * n2))
            if kind == "summed":
                acc += g                                                      # one step at the end of the sweep
            else:
                w = w + gamma * g if kind == "uphill" else w - gamma * g
        if kind == "summed":
            w = w - gamma * acc
        return z, w, tot / len(positions)
    return bad


@pytest.mark.parametrize("kind,pin", [
    ("old_patch", "test_epie_sweep_probe_step_at_the_updated_patch"),
    ("no_conj", "test_epie_sweep_probe_step_projects_the_probe"),
    ("uphill", "test_epie_sweep_probe_step_projects_the_probe"),
    ("summed", "test_epie_sweep_updates_the_probe_after_every_position"),
])
def test_epie_sweep_mistakes(monkeypatch, kind, pin):
    monkeypatch.setattr(pie, "epie_sweep", _bad_epie_sweep(kind))
    fails(getattr(t_pie, pin))
