"""Pins of the training-side oracle (oracle/train.py) against what fixes it from outside: torch's
own Adam and autograd (library routines), closed forms of the first Adam step and of the
learning-rate schedule, and hand-built density-control cases whose outcome follows from the rules
by inspection."""
import math

import numpy as np
import pytest

from oracle import train as ot

torch = pytest.importorskip("torch")


def _set(n, nb=16, seed=0):
    rng = np.random.default_rng(seed)
    raw = dict(means=rng.normal(0, 1, (n, 3)), scales=rng.uniform(-5, -1, (n, 3)), quats=rng.normal(0, 1, (n, 4)),
               betas=rng.uniform(-1.5, 4, n), opacities=rng.normal(0, 2, n), shs=rng.normal(0, 0.3, (n, nb, 3)))
    zeros = {k: np.zeros_like(a) for k, a in raw.items()}
    return raw, zeros, {k: a.copy() for k, a in zeros.items()}


def _grads(n, nb=16, seed=1):
    rng = np.random.default_rng(seed)
    return dict(means=rng.normal(0, 1e-3, (n, 3)), scales=rng.normal(0, 1e-2, (n, 3)),
                quats=rng.normal(0, 1e-3, (n, 4)), betas=rng.normal(0, 1e-3, n), opacities=rng.normal(0, 1e-2, n),
                shs=rng.normal(0, 1e-3, (n, nb, 3)))


def test_adam_matches_torch_adam_with_autograd_chain_rule():
    """Five steps on every group against torch.optim.Adam, with the raw gradients taken by torch
    autograd through the activations (exp, sigmoid, +2) instead of the oracle's chain rule."""
    n, nb = 7, 16
    raw, m, v = _set(n, nb)
    hp = ot.ADAM_DEFAULTS
    tr = {k: torch.tensor(a, dtype=torch.float64, requires_grad=True) for k, a in raw.items()}
    groups = [{"params": [tr[k]], "lr": hp["lr_" + k]} for k in ("means", "scales", "quats", "betas", "opacities")]
    # SH: DC and the rest at different rates -> optimise them as two views through a mask
    dc_mask = torch.zeros((n, nb, 3), dtype=torch.float64)
    dc_mask[:, 0, :] = 1.0
    sh_a = torch.tensor(raw["shs"] * dc_mask.numpy(), requires_grad=True)
    sh_b = torch.tensor(raw["shs"] * (1 - dc_mask.numpy()), requires_grad=True)
    groups += [{"params": [sh_a], "lr": hp["lr_sh_dc"]}, {"params": [sh_b], "lr": hp["lr_sh_rest"]}]
    opt = torch.optim.Adam(groups, betas=(hp["beta1"], hp["beta2"]), eps=hp["eps"])
    for step in range(1, 6):
        g = _grads(n, nb, seed=10 + step)
        raw, m, v, phys = ot.adam_step(raw, m, v, g, step)
        opt.zero_grad()
        phys_t = [tr["means"], torch.exp(tr["scales"]), tr["quats"], tr["betas"] + 2.0, torch.sigmoid(tr["opacities"])]
        loss = sum((p * torch.tensor(g[k])).sum() for p, k in zip(phys_t, ("means", "scales", "quats", "betas",
                                                                              "opacities")))
        loss = loss + ((sh_a * dc_mask + sh_b * (1 - dc_mask)) * torch.tensor(g["shs"])).sum()
        loss.backward()
        opt.step()
        for k in ("means", "scales", "quats", "betas", "opacities"):
            np.testing.assert_allclose(raw[k], tr[k].detach().numpy(), rtol=1e-12, atol=1e-14)
        sh = (sh_a * dc_mask + sh_b * (1 - dc_mask)).detach().numpy()
        np.testing.assert_allclose(raw["shs"], sh, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(phys["scales"], np.exp(raw["scales"]), rtol=1e-15)
        np.testing.assert_allclose(phys["opacities"], 1 / (1 + np.exp(-raw["opacities"])), rtol=1e-15)
        np.testing.assert_allclose(phys["betas"], raw["betas"] + 2.0, rtol=0, atol=1e-15)


def test_first_adam_step_moves_each_element_by_its_learning_rate():
    """At step 1 the bias-corrected ratio is g / |g|: every element with |g| >> eps moves by -lr sign(g)."""
    n = 5
    raw, m, v = _set(n)
    g = _grads(n)
    new, _, _, _ = ot.adam_step(raw, m, v, g, 1)
    gr = ot.raw_gradient(raw, g)
    hp = ot.ADAM_DEFAULTS
    def check(d, lr, g):  # |d + lr sign(g)| <= lr (eps / |g| + rounding)
        assert np.all(np.abs(d + lr * np.sign(g)) <= lr * (hp["eps"] / np.abs(g) + 1e-11))

    for k in ("means", "scales", "quats", "betas", "opacities"):
        check(new[k] - raw[k], hp["lr_" + k], gr[k])
    d = (new["shs"] - raw["shs"]).reshape(n, -1)
    g = gr["shs"].reshape(n, -1)
    check(d[:, :3], hp["lr_sh_dc"], g[:, :3])
    check(d[:, 3:], hp["lr_sh_rest"], g[:, 3:])


def test_position_learning_rate_schedule():
    """App. B.2: 1.6e-4 at the start, 1.6e-6 from step 30000 on, log-linear in between."""
    assert ot.position_lr(0) == pytest.approx(1.6e-4, rel=1e-15)
    assert ot.position_lr(30000) == pytest.approx(1.6e-6, rel=1e-12)
    assert ot.position_lr(40000) == pytest.approx(1.6e-6, rel=1e-12)
    assert ot.position_lr(15000) == pytest.approx(1.6e-5, rel=1e-12)        # geometric mean
    assert ot.position_lr(7500) == pytest.approx(1.6e-4 * 10 ** -0.5, rel=1e-12)
    # with a warm-up, step 0 starts at delay_mult times the rate and reaches it at delay_steps
    assert ot.position_lr(0, delay_steps=1000) == pytest.approx(0.01 * 1.6e-4, rel=1e-12)
    assert ot.position_lr(1000, delay_steps=1000) == pytest.approx(ot.position_lr(1000), rel=1e-12)


def test_densify_stats_by_hand():
    inter = np.zeros((3, 10))
    inter[:, 0] = [0.3, -1.0, 2.0]
    inter[:, 1] = [0.4, 0.0, 5.0]
    acc, cnt = ot.densify_stats([1, 0, 7], inter, 2, 2)         # W/2 = H/2 = 1: plain norms
    np.testing.assert_allclose(acc, [0.5, 0.0, math.hypot(2, 5)], rtol=1e-15)
    assert list(cnt) == [1, 0, 1]
    acc, cnt = ot.densify_stats([1, 1, 0], inter, 8, 4, acc, cnt)  # x scaled by 4, y by 2
    np.testing.assert_allclose(acc, [0.5 + math.hypot(1.2, 0.8), 4.0, math.hypot(2, 5)], rtol=1e-15)
    assert list(cnt) == [2, 1, 1]


def _rows(n, nb=1):
    raw = dict(means=np.zeros((n, 3)), scales=np.full((n, 3), math.log(0.005)), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
               betas=np.zeros(n), opacities=np.zeros(n), shs=np.zeros((n, nb, 3)))
    raw["means"][:, 0] = np.arange(n)   # row tag
    m = {k: np.full_like(a, 0.25) for k, a in raw.items()}
    v = {k: np.full_like(a, 0.5) for k, a in raw.items()}
    return raw, m, v


def test_density_control_by_hand():
    """Row 0 quiet (kept), 1 high gradient and small (cloned), 2 high gradient and large (split),
    3 transparent (pruned), 4 sharp beta = 0.3 (shape-pruned), 5 large and quiet but beyond the
    world-size limit (pruned), 6 split whose children stay beyond the limit (gone)."""
    raw, m, v = _rows(7)
    raw["scales"][2] = np.log([0.05, 0.02, 0.03])
    raw["quats"][2] = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]   # 90 degrees about z
    raw["opacities"][3] = math.log(0.004 / 0.996)
    raw["betas"][4] = 0.3 - 2.0
    raw["scales"][5] = math.log(0.2)
    raw["scales"][6] = math.log(0.5)
    accum = np.array([1e-4, 4e-3, 4e-3, 0.0, 0.0, 0.0, 9e-3])
    count = np.array([1, 10, 10, 3, 0, 2, 10])
    xi = np.zeros((7, 2, 3))
    xi[2, 0] = [1.0, 2.0, -1.0]
    xi[2, 1] = [-0.5, 0.0, 3.0]
    out, om, ov, d = ot.density_control(raw, m, v, accum, count, xi, extent=1.0, min_beta=0.5, max_world=0.1)
    assert list(out["means"][:, 0].round(6)) == [0.0, 1.0, 1.0, 2.0 - 2 * 0.02, 2.0 + 0.0]
    # children of row 2: R = rotation by 90 degrees about z maps (x, y, z) -> (-y, x, z)
    np.testing.assert_allclose(out["means"][3], [2.0 - 0.02 * 2.0, 0.05 * 1.0, 0.03 * -1.0], atol=1e-15)
    np.testing.assert_allclose(out["means"][4], [2.0 - 0.0, 0.05 * -0.5, 0.03 * 3.0], atol=1e-15)
    np.testing.assert_allclose(np.exp(out["scales"][3:5]), np.tile([0.05, 0.02, 0.03], (2, 1)) / 1.6, rtol=1e-15)
    np.testing.assert_allclose(out["quats"][3], raw["quats"][2], rtol=0)
    # moments: the kept rows 0 and 1 keep theirs, the clone and the children start from zero
    for k in ot.GROUPS:
        assert np.all(om[k][:2] == 0.25) and np.all(ov[k][:2] == 0.5)
        assert np.all(om[k][2:] == 0) and np.all(ov[k][2:] == 0)
    assert list(np.nonzero(d["keep"])[0]) == [0, 1] and list(np.nonzero(d["clone"])[0]) == [1]
    assert list(np.nonzero(d["split"])[0]) == [2, 6] and list(np.nonzero(d["child"])[0]) == [2]


def test_density_control_counts_and_prune_only():
    raw, m, v = _set(200, nb=4, seed=3)
    raw["betas"][:10] = 0.4 - 2.0     # shape-pruned
    raw["opacities"][10:20] = -6.0    # below 0.005
    rng = np.random.default_rng(4)
    accum = rng.exponential(3e-4, 200) * 5
    count = rng.integers(0, 6, 200)
    xi = rng.standard_normal((200, 2, 3))
    out, _, _, d = ot.density_control(raw, m, v, accum, count, xi, extent=4.0, min_beta=0.5)
    assert out["means"].shape[0] == d["keep"].sum() + d["clone"].sum() + 2 * d["child"].sum()
    assert d["clone"].sum() > 0 and d["child"].sum() > 0 and (~d["keep"] & ~d["split"]).sum() > 0
    # with no densification (threshold above every gradient) only the prune rules act
    out2, _, _, d2 = ot.density_control(raw, m, v, accum, count, xi, grad_threshold=1e9, extent=4.0, min_beta=0.5)
    kappa = 1 / (1 + np.exp(-raw["opacities"]))
    want = (kappa >= 0.005) & (raw["betas"] + 2 >= 0.5)
    assert np.array_equal(d2["keep"], want) and out2["means"].shape[0] == want.sum()


def test_resets():
    raw, m, v = _set(50, seed=5)
    m = {k: a + 1 for k, a in m.items()}
    r, mm, vv = ot.reset_opacity(raw, m, v)
    k = 1 / (1 + np.exp(-r["opacities"]))
    k0 = 1 / (1 + np.exp(-raw["opacities"]))
    np.testing.assert_allclose(k, np.minimum(k0, 0.01), rtol=1e-12)
    assert np.all(mm["opacities"] == 0) and np.all(mm["means"] == 1)
    r, mm, vv = ot.reset_shape(raw, m, v)
    assert np.all(r["betas"] + 2.0 == 2.0) and np.all(mm["betas"] == 0) and np.all(mm["scales"] == 1)
