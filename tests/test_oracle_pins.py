"""Pins for the FP64 oracle: each test checks it against something other than itself
(closed forms, textbook special cases, library routines on special cases,
invariants, finite differences).  CPU only."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from helpers import Y00, axis_camera, make_scene, random_small_scene, rel_err
from paper_2402_10128_gb300 import scenes

# the kernels take their parameters as float32; closed forms use the same values
RHO32 = float(np.float32(0.1))
DIL32 = float(np.float32(0.3))
AMAX32, AMIN32, TMIN32 = (float(np.float32(v)) for v in (0.99, 1.0 / 255.0, 1e-4))
GOLDEN = __file__.replace("test_oracle_pins.py", "golden/paper_constants.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split("=")
            out[k.strip()] = float(v)
    return out


# ---------------------------------------------------------------- key-path exp2/log2
def test_key_exp2_log2_match_libm_within_ulps():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-60, 60, 2000), rng.uniform(-1, 1, 2000), [0.0, 1.0, -1.0, 0.5, 20.25]])
    for x in xs.astype(np.float32):
        got = np.float32(oracle.key_exp2(float(x)))
        ref = np.float32(2.0 ** float(x))
        ulp = np.spacing(ref)
        assert abs(float(got) - float(ref)) <= 4 * ulp, (x, got, ref)
    ys = np.concatenate([np.exp(rng.uniform(-20, 20, 3000)), [1.0, 2.0, 0.5, 3.0, 255.0]]).astype(np.float32)
    for y in ys:
        got = oracle.key_log2(float(y))
        ref = math.log2(float(y))
        assert abs(got - ref) <= 4 * np.spacing(np.float32(max(abs(ref), 1.0))), (y, got, ref)
    assert oracle.key_exp2(0.0) == 1.0 and oracle.key_exp2(3.0) == 8.0 and oracle.key_log2(1.0) == 0.0


# ---------------------------------------------------------------- shape modification
def test_phi_bar_fixed_points_and_symmetry():
    g = _golden()
    assert oracle.phi_bar(2.0, rho=g["rho"])[0] == g["phi_bar_at_beta_2"]      # Sec. 4.2: exactly 1 at beta=2
    x = np.linspace(0.0, 30.0, 301)
    s = oracle.phi_bar(2.0 + x) + oracle.phi_bar(2.0 - x)                       # sigmoid identity
    assert np.max(np.abs(s - 2.0)) < 1e-15
    assert np.all(oracle.phi_bar(np.linspace(0.01, 50, 500), rho=0.0) == 1.0)  # rho=0 -> Gaussian for any beta
    v = oracle.phi_bar(np.linspace(0.01, 50, 500))
    assert np.all(np.diff(v) > 0) and np.all(v > 0) and np.all(v < 2)


def test_phi_exact_closed_forms():
    # Gamma(3/2)/Gamma(1/2) = 1/2, Gamma(3)/Gamma(1) = 2, Gamma(3/4)/Gamma(1/4) at beta=4
    assert abs(oracle.phi_exact(2.0)[0] - 0.5) < 1e-15
    assert abs(oracle.phi_exact(1.0)[0] - 2.0) < 1e-14
    assert abs(oracle.phi_exact(4.0)[0] - math.gamma(0.75) / math.gamma(0.25)) < 1e-14


def _phi_ref(beta, phi_mode, rho=RHO32):
    """The scale modification written from Sec. 4.2 with the standard library's Gamma function:
    phi_bar_rho (Eq. approx); 2 Gamma(3/b)/Gamma(1/b) (Eq. probablity, normalised to 1 at b = 2);
    its square root (the ratio read as one of variances, Eq. effective)."""
    if phi_mode == oracle.PHI_APPROX:
        return 2.0 / (1.0 + math.exp(-rho * (beta - 2.0)))
    r = 2.0 * math.gamma(3.0 / beta) / math.gamma(1.0 / beta)
    return r if phi_mode == oracle.PHI_EXACT else math.sqrt(r)


def test_digamma_special_values_and_recurrence():
    gamma_e = 0.57721566490153286  # Euler-Mascheroni constant: psi(1) = -gamma
    assert abs(oracle.digamma(1.0) + gamma_e) < 1e-14
    assert abs(oracle.digamma(0.5) + gamma_e + 2 * math.log(2.0)) < 1e-14   # psi(1/2) = -gamma - 2 ln 2
    for n in range(1, 25):                                                     # psi(n+1) = H_n - gamma
        h = sum(1.0 / k for k in range(1, n + 1))
        assert abs(oracle.digamma(n + 1.0) - (h - gamma_e)) < 1e-14 * max(1.0, h)
    rng = np.random.default_rng(30)
    for x in np.exp(rng.uniform(math.log(0.02), math.log(200.0), 200)):
        # psi(x + 1) - psi(x) = 1/x, and psi is the slope of ln Gamma (central differences of libm)
        assert abs(oracle.digamma(x + 1) - oracle.digamma(x) - 1 / x) < 1e-12 * max(1.0, 1 / x)
        h = 1e-5 * x
        fd = (math.lgamma(x + h) - math.lgamma(x - h)) / (2 * h)
        assert abs(oracle.digamma(x) - fd) < 1e-7 * max(1.0, abs(fd))


def test_key_lgamma_matches_the_library():
    """The key path's FP32 ln Gamma (shift to z >= 4, Stirling's series) against libm's."""
    xs = np.concatenate([np.exp(np.linspace(math.log(1 / 64), math.log(64.0), 400)), [0.5, 1.0, 2.0, 3.0, 8.0]])
    for x in xs.astype(np.float32):
        got, ref = oracle.key_lgamma(float(x)), math.lgamma(float(x))
        assert abs(got - ref) <= 2.5e-6 * max(1.0, abs(ref)), (x, got, ref)


@pytest.mark.parametrize("phi_mode", [0, 1, 2])
def test_key_phi_matches_the_gamma_ratio(phi_mode):
    """The key path's FP32 scale modification against Sec. 4.2 written with math.gamma."""
    for b in np.exp(np.linspace(math.log(0.4), math.log(32.0), 300)).astype(np.float32):
        got, ref = oracle.key_phi(float(b), RHO32, phi_mode), _phi_ref(float(b), phi_mode)
        assert abs(got - ref) <= 4e-6 * ref, (b, got, ref)


def test_phi_exact_normalised_closed_forms():
    g = _golden()
    P1 = dict(phi_mode=oracle.PHI_EXACT)
    P2 = dict(phi_mode=oracle.PHI_EXACT_VARIANCE)
    phi = lambda b, p: oracle.phi_mod(b, p)[0][0]
    # 1 at beta = 2 (Sec. 4.2, after Eq. approx; Fig. approximation caption), in both readings
    assert abs(phi(2.0, P1) - g["phi_bar_at_beta_2"]) < 1e-15 and abs(phi(2.0, P2) - 1.0) < 1e-15
    assert abs(phi(1.0, P1) - 4.0) < 1e-14            # 2 Gamma(3) / Gamma(1)
    assert abs(phi(0.5, P1) - 240.0) < 1e-11          # 2 Gamma(6) / Gamma(2) = 2 * 5!
    assert abs(phi(3.0, P1) - 2.0 / math.gamma(1 / 3)) < 1e-14
    assert abs(phi(1.0, P2) - 2.0) < 1e-14
    # beta -> infinity: Gamma(3/b)/Gamma(1/b) -> 1/3 (the box), so phi_n -> 2/3
    assert abs(phi(1e7, P1) - 2.0 / 3.0) < 1e-6
    # the normalisation of the unnormalised ratio printed in Eq. probablity
    for b in (0.7, 1.3, 2.9, 6.0):
        assert abs(phi(b, P1) - 2.0 * oracle.phi_exact(b)[0]) < 1e-13 * phi(b, P1)


@pytest.mark.parametrize("phi_mode", [0, 1, 2])
def test_phi_derivative_by_finite_differences(phi_mode):
    """d phi / d beta carried by the oracle's dual numbers (digamma for the exact forms) against
    central differences of its value (libm's lgamma)."""
    params = dict(phi_mode=phi_mode)
    b = np.exp(np.linspace(math.log(0.4), math.log(24.0), 60))
    _, d = oracle.phi_mod(b, params)
    h = 1e-6 * b
    fd = (oracle.phi_mod(b + h, params)[0] - oracle.phi_mod(b - h, params)[0]) / (2 * h)
    assert np.all(np.abs(d - fd) <= 1e-6 * np.maximum(np.abs(fd), 1e-3))
    if phi_mode == oracle.PHI_EXACT:
        # at beta = 1: 4 (psi(1) - 3 psi(3)) with psi(1) = -gamma, psi(3) = 3/2 - gamma: 4 (2 gamma - 9/2)
        gamma_e = 0.57721566490153286
        assert abs(oracle.phi_mod(1.0, params)[1][0] - 4 * (2 * gamma_e - 4.5)) < 1e-12


def test_eta_bounds_arithmetic():
    g = _golden()
    assert abs((4 - math.pi) / math.pi - g["eta_square_larger"]) < 5e-5
    assert abs((math.pi - 2) / math.pi - g["eta_circle_larger"]) < 5e-5


# ---------------------------------------------------------------- spherical harmonics
def _sphere_quadrature(nz=16, nphi=32):
    z, wz = np.polynomial.legendre.leggauss(nz)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    W = np.outer(wz, np.full(nphi, 2 * np.pi / nphi))
    r = np.sqrt(1 - Z ** 2)
    d = np.stack([r * np.cos(P), r * np.sin(P), Z], -1).reshape(-1, 3)
    return d, W.reshape(-1)


def test_sh_orthonormal_by_quadrature():
    d, w = _sphere_quadrature()
    Y = oracle.sh_basis(3, d)
    G = (Y * w[:, None]).T @ Y
    assert np.max(np.abs(G - np.eye(16))) < 1e-12


def test_sh_addition_theorem_and_parity():
    rng = np.random.default_rng(1)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(3, d)
    Yn = oracle.sh_basis(3, -d)
    for l in range(4):
        sl = slice(l * l, (l + 1) ** 2)
        assert np.max(np.abs((Y[:, sl] ** 2).sum(1) - (2 * l + 1) / (4 * np.pi))) < 1e-12
        assert np.max(np.abs(Yn[:, sl] - (-1) ** l * Y[:, sl])) < 1e-12
    assert abs(Y[0, 0] - Y00) < 1e-15
    # Y_{1,0} along +z = sqrt(3/4pi); Y_{1,1} ~ -x (Condon-Shortley phase)
    e = oracle.sh_basis(1, np.array([[0.0, 0, 1], [1.0, 0, 0]]))
    assert abs(e[0, 2] - math.sqrt(3 / (4 * math.pi))) < 1e-15
    assert abs(e[1, 3] + math.sqrt(3 / (4 * math.pi))) < 1e-15


# ---------------------------------------------------------------- projection
@pytest.mark.parametrize("phi_mode", [0, 1, 2])
def test_isotropic_on_axis_projection_closed_form(phi_mode):
    cam = axis_camera(64, 64)
    params = dict(phi_mode=phi_mode)
    for beta in (2.0, 0.7, 5.0):
        s, z = 0.125 if phi_mode == 0 else 0.0625, 4.0
        sc = make_scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [beta], [0.8], rgb=[[0.3, 0.6, 0.9]])
        pr = oracle.project(sc, cam, params)[0]
        b32, dil32 = (float(np.float32(v)) for v in (beta, 0.3))
        phi = _phi_ref(b32, phi_mode)
        var = (cam.fx * phi * s / z) ** 2 + dil32
        assert abs(pr[0] - cam.cx) < 1e-12 and abs(pr[1] - cam.cy) < 1e-12
        assert abs(pr[5] - var) < 1e-12 * var and abs(pr[6]) < 1e-15 and abs(pr[7] - var) < 1e-12 * var
        assert abs(pr[2] - 1 / var) < 1e-12 / var and abs(pr[4] - 1 / var) < 1e-12 / var
        np.testing.assert_allclose(pr[8:11], [0.3, 0.6, 0.9], atol=1e-6)
        k = oracle.keys(sc, cam, params)
        # FP32 key path: phi_n carries up to 2e-6 relative error (its Gamma ratio in FP32), twice that in var
        np.testing.assert_allclose(k["cov2d"][0], [var, 0, var], rtol=1e-6 if phi_mode == 0 else 5e-6, atol=1e-6)
        np.testing.assert_allclose(k["mean2d"][0], [cam.cx, cam.cy], rtol=0, atol=1e-4)


def test_isotropic_rotation_invariance():
    cam = axis_camera(64, 64)
    rng = np.random.default_rng(2)
    q = rng.standard_normal((20, 4))
    m = np.tile([[0.3, -0.2, 3.0]], (20, 1))
    sc = make_scene(m, np.full((20, 3), 0.07), q, np.full(20, 1.5), np.full(20, 0.5), rgb=np.full((20, 3), 0.5))
    pr = oracle.project(sc, cam)
    assert np.max(np.abs(pr[:, 5:8] - pr[0, 5:8])) < 1e-11


def _complex_step_jacobian(cam, t):
    """Jacobian of the pinhole map at camera-space point t, by complex step (exact)."""
    h = 1e-30
    J = np.zeros((2, 3))
    for k in range(3):
        tt = np.asarray(t, np.complex128).copy()
        tt[k] += 1j * h
        u = cam.fx * tt[0] / tt[2] + cam.cx
        v = cam.fy * tt[1] / tt[2] + cam.cy
        J[:, k] = [u.imag / h, v.imag / h]
    return J


def test_anisotropic_ewa_matches_textbook():
    cam = scenes.look_at((0.5, -0.3, -4.0), (0.1, 0.0, 0.0), (0.0, -1.0, 0.0), 96, 80, 55.0)
    rng = np.random.default_rng(3)
    n = 12
    m = rng.uniform(-0.8, 0.8, (n, 3))
    s = rng.uniform(0.03, 0.3, (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    b = rng.uniform(0.5, 6, n)
    sc = make_scene(m, s, q, b, np.full(n, 0.7), rgb=np.full((n, 3), 0.5))
    pr = oracle.project(sc, cam)
    V = cam.viewmat.astype(np.float64)
    for i in range(n):
        mu = sc.means[i].astype(np.float64)
        t = V[:3, :3] @ mu + V[:3, 3]
        Rq = Rotation.from_quat(np.r_[sc.quats[i, 1:], sc.quats[i, 0]].astype(np.float64)).as_matrix()
        phi = 2.0 / (1.0 + math.exp(-RHO32 * (float(sc.betas[i]) - 2.0)))
        Sig = Rq @ np.diag((phi * sc.scales[i].astype(np.float64)) ** 2) @ Rq.T
        J = _complex_step_jacobian(cam, t)
        cov = J @ V[:3, :3] @ Sig @ V[:3, :3].T @ J.T + DIL32 * np.eye(2)
        np.testing.assert_allclose(pr[i, [5, 6, 7]], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-11, atol=1e-12)
        uv = [cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy]
        np.testing.assert_allclose(pr[i, :2], uv, rtol=1e-13)


# ---------------------------------------------------------------- falloff
@pytest.mark.parametrize("beta,phi_mode", [(1.0, 0), (2.0, 0), (0.6, 0), (3.5, 0), (1.0, 1), (3.5, 1), (0.8, 2)])
def test_lone_splat_is_the_1d_gef(beta, phi_mode):
    """A lone isotropic splat on the optical axis, bg = 0: along the centre row the
    pixel value is rgb * min(0.99, A exp(-(|x-mu|/alpha)^beta)) with A = kappa and
    alpha = sigma' 2^(1/beta) (Eq. gef); beta=1 is Laplace-shaped, beta=2 Gaussian."""
    W = 64
    cam = axis_camera(W, W)
    s, z, kappa = 0.0625, 3.0, 0.875
    rgb = np.array([0.25, 0.5, 1.0])
    sc = make_scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [beta], [kappa], rgb=[rgb])
    out = oracle.render(sc, cam, params=dict(phi_mode=phi_mode))
    b32, dil32 = (float(np.float32(v)) for v in (beta, 0.3))
    rgb = Y00 * sc.shs[0, 0].astype(np.float64) + 0.5
    phi = _phi_ref(b32, phi_mode)
    sigma = math.sqrt((cam.fx * phi * s / z) ** 2 + dil32)
    alpha_scale = sigma * 2.0 ** (1.0 / b32)
    row = W // 2  # pixel centre y = 32.5, mean y = 32 -> offset 0.5
    for x in range(W):
        dx, dy = x + 0.5 - cam.cx, row + 0.5 - cam.cy
        r = math.hypot(dx, dy)
        a = min(AMAX32, kappa * math.exp(-((r / alpha_scale) ** b32)))
        expect = rgb * a if a >= AMIN32 else np.zeros(3)
        np.testing.assert_allclose(out["img"][:, row, x], expect, rtol=1e-12, atol=1e-14)
    assert out["img"][2, row, W // 2] > 0.5


def test_two_splat_compositing_closed_form():
    W = 32
    cam = axis_camera(W, W, bg=(0.1, 0.2, 0.3))
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.4])
    sc = make_scene([[0, 0, 3.0], [0.0, 0, 5.0]], [[0.25] * 3, [0.375] * 3], [[1, 0, 0, 0]] * 2,
                    [2.0, 2.0], [0.6, 0.7], rgb=[c1, c2])
    pr = oracle.project(sc, cam)
    out = oracle.render(sc, cam)
    c1, c2 = (Y00 * sc.shs[i, 0].astype(np.float64) + 0.5 for i in range(2))
    for (x, y) in [(16, 16), (15, 17), (18, 14)]:
        d = np.array([x + 0.5 - cam.cx, y + 0.5 - cam.cy])
        al = []
        for i in range(2):
            C = np.array([[pr[i, 2], pr[i, 3]], [pr[i, 3], pr[i, 4]]])
            al.append(min(AMAX32, float(sc.opacities[i]) * math.exp(-0.5 * d @ C @ d)))
        assert min(al) > 0.05
        bg = np.array(cam.bg, np.float32).astype(np.float64)
        expect = c1 * al[0] + c2 * al[1] * (1 - al[0]) + bg * (1 - al[0]) * (1 - al[1])
        np.testing.assert_allclose(out["img"][:, y, x], expect, rtol=1e-13)
        assert abs(out["T"][y, x] - (1 - al[0]) * (1 - al[1])) < 1e-15


def _gaussian_reference(scene, cam, scale_mult=None, dilation=DIL32):
    """Independent pure-Gaussian splat renderer (exp(-q/2), no shape parameter) written
    with scipy rotations and a complex-step Jacobian; SH degree 0 only."""
    V = cam.viewmat.astype(np.float64)
    prims = []
    for i in range(scene.n):
        mu = scene.means[i].astype(np.float64)
        t = V[:3, :3] @ mu + V[:3, 3]
        if t[2] <= cam.znear:
            continue
        q = scene.quats[i].astype(np.float64)
        Rq = Rotation.from_quat(np.r_[q[1:], q[0]]).as_matrix()
        s = scene.scales[i].astype(np.float64) * (1.0 if scale_mult is None else scale_mult[i])
        Sig = Rq @ np.diag(s ** 2) @ Rq.T
        J = _complex_step_jacobian(cam, t)
        cov = J @ V[:3, :3] @ Sig @ V[:3, :3].T @ J.T + dilation * np.eye(2)
        rgb = np.maximum(0.0, Y00 * scene.shs[i, 0].astype(np.float64) + 0.5)
        uv = np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
        prims.append((np.float32(t[2]), i, uv, np.linalg.inv(cov), rgb, float(scene.opacities[i])))
    prims.sort(key=lambda p: (p[0], p[1]))
    W, H = cam.width, cam.height
    ys, xs = np.mgrid[0:H, 0:W]
    P = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5], 1)
    T = np.ones(P.shape[0])
    C = np.zeros((3, P.shape[0]))
    done = np.zeros(P.shape[0], bool)
    for _, _, uv, conic, rgb, kappa in prims:
        d = P - uv
        qv = np.einsum("pi,ij,pj->p", d, conic, d)
        a = np.minimum(AMAX32, kappa * np.exp(-0.5 * qv))
        use = (~done) & (a >= AMIN32)
        Tn = T * (1 - a)
        stop = use & (Tn < TMIN32)
        done |= stop
        use &= ~stop
        C += np.where(use, rgb[:, None] * a * T, 0.0)
        T = np.where(use, Tn, T)
    bg = np.asarray(cam.bg, np.float64)[:, None]
    return (C + T * bg).reshape(3, H, W), T.reshape(H, W)


def test_beta2_equals_independent_gaussian_renderer():
    sc = random_small_scene(25, seed=4, beta_range=(2.0, 2.0))
    cam = axis_camera(48, 40)
    ref, Tref = _gaussian_reference(sc, cam)
    for mode in (oracle.MODE_GEF, oracle.MODE_PAPER_APPROX):
        out = oracle.render(sc, cam, params=dict(mode=mode))
        assert np.max(np.abs(out["img"] - ref)) < 1e-10
        assert np.max(np.abs(out["T"] - Tref)) < 1e-10


def test_beta2_scale_modifications_agree():
    """At beta = 2 every form of the modification is 1 (Sec. 4.2), so the images agree."""
    sc = random_small_scene(25, seed=4, beta_range=(2.0, 2.0))
    cam = axis_camera(48, 40)
    ref = oracle.render(sc, cam)["img"]
    for pm in (oracle.PHI_EXACT, oracle.PHI_EXACT_VARIANCE):
        assert np.max(np.abs(oracle.render(sc, cam, params=dict(phi_mode=pm))["img"] - ref)) < 1e-12


def test_exact_phi_paper_form_is_the_scaled_gaussian():
    """With the exact modification, the paper's Gaussian-form rasterizer is the Gaussian with its
    scales times 2 Gamma(3/b)/Gamma(1/b) (Eq. probablity), written here with math.gamma."""
    sc = random_small_scene(25, seed=5, beta_range=(1.0, 9.0))
    cam = axis_camera(48, 40)
    mult = np.array([_phi_ref(float(b), oracle.PHI_EXACT) for b in sc.betas.astype(np.float64)])
    ref, _ = _gaussian_reference(sc, cam, scale_mult=mult)
    out = oracle.render(sc, cam, params=dict(mode=oracle.MODE_PAPER_APPROX, phi_mode=oracle.PHI_EXACT))
    assert np.max(np.abs(out["img"] - ref)) < 1e-10


def test_rho0_paper_form_is_gaussian_for_any_beta():
    sc = random_small_scene(25, seed=5, beta_range=(0.3, 9.0))
    cam = axis_camera(48, 40)
    ref, _ = _gaussian_reference(sc, cam)
    out = oracle.render(sc, cam, params=dict(mode=oracle.MODE_PAPER_APPROX, rho=0.0))
    assert np.max(np.abs(out["img"] - ref)) < 1e-10
    # and with rho = 0.1 the paper form is the Gaussian with scales times phi_bar(beta) (Eq. approx)
    phi = 2.0 / (1.0 + np.exp(-(RHO32 * sc.betas.astype(np.float64) - 2.0 * RHO32)))
    ref2, _ = _gaussian_reference(sc, cam, scale_mult=phi)
    out2 = oracle.render(sc, cam, params=dict(mode=oracle.MODE_PAPER_APPROX))
    assert np.max(np.abs(out2["img"] - ref2)) < 1e-10


# ---------------------------------------------------------------- compositing invariants
def test_transmittance_bounds_and_monotone():
    sc, cam = scenes.tiny_workload()
    out = oracle.render(sc, cam)
    assert out["T"].min() >= 1e-4 and out["T"].max() <= 1.0
    # T is non-increasing as primitives are added behind: drop the farthest half
    k = oracle.keys(sc, cam)
    order = np.argsort(k["depth_key"], kind="stable")
    front = np.sort(order[: sc.n // 2])
    out_front = oracle.render(sc.subset(front), cam)
    assert np.all(out["T"] <= out_front["T"] + 1e-15)


def test_permutation_invariance():
    sc, cam = scenes.tiny_workload()
    perm = np.random.default_rng(7).permutation(sc.n)
    a = oracle.render(sc, cam)["img"]
    b = oracle.render(sc.subset(perm), cam)["img"]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["tiny", "ragged_lowbeta", "ragged_paper_form"])
def test_tiled_equals_brute_force(case):
    if case == "tiny":
        sc, cam = scenes.tiny_workload()
        params = None
    else:
        sc = scenes.cube_scene(300, seed=11, beta_range=(0.3, 16.0), beta_log=True, scale_range=(0.02, 0.2))
        cam = scenes.tiny_camera(45, 37)
        params = dict(mode=oracle.MODE_PAPER_APPROX) if case == "ragged_paper_form" else None
    a = oracle.render(sc, cam, params=params)
    b = oracle.render(sc, cam, params=params, tiled=True)
    assert np.array_equal(a["img"], b["img"]) and np.array_equal(a["T"], b["T"])


def test_key_list_structure():
    sc, cam = scenes.tiny_workload()
    k = oracle.keys(sc, cam)
    kk, vv = oracle.sorted_keys(sc, cam, key_info=k)
    assert kk.size == int(k["touched"].sum())
    assert np.all(np.diff(kk.astype(np.uint64)) >= 0) or np.all(kk[1:] >= kk[:-1])
    tiles = (kk >> np.uint64(32)).astype(np.int64)
    tx = (cam.width + 15) // 16
    r = k["rect"][vv]
    assert np.all((tiles % tx >= r[:, 0]) & (tiles % tx < r[:, 2]) & (tiles // tx >= r[:, 1]) & (tiles // tx < r[:, 3]))
    assert np.all((kk & np.uint64(0xFFFFFFFF)).astype(np.uint32) == k["depth_key"][vv])
    # equal keys keep ascending primitive index
    same = kk[1:] == kk[:-1]
    assert np.all(vv[1:][same] > vv[:-1][same])
    # depth key is the float32 bit pattern of a positive depth
    vis = k["touched"] > 0
    d = k["depth_key"][vis].view(np.float32)
    assert np.all(d > 0.2)


def _qmin_over_box(conic, u, v, x0, x1, y0, y1):
    """min of q(d) = d^T conic d, d = (x - u, y - v), over the box [x0,x1] x [y0,y1] (FP64): zero if
    the centre is inside, else the smallest of the four edges' 1D minima (closed form, clamped)."""
    if x0 <= u <= x1 and y0 <= v <= y1:
        return 0.0
    A, B, C = conic
    best = math.inf
    for x in (x0, x1):            # vertical edges: minimise over y
        dx = x - u
        dy = min(max(-B * dx / C, y0 - v), y1 - v)
        best = min(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    for y in (y0, y1):            # horizontal edges: minimise over x
        dy = y - v
        dx = min(max(-B * dy / A, x0 - u), x1 - u)
        best = min(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    return best


@pytest.mark.parametrize("which", ["tiny", "wide_beta"])
def test_tile_lists_follow_the_extent_ellipse(which):
    """Each primitive's tiles are exactly those its extent ellipse {d^T cov^-1 d <= q_lim} meets,
    up to the 1e-2 px horizontal margin: checked against a geometric test written independently of
    the row-span formula (the minimum of the quadratic form over each tile's box)."""
    if which == "tiny":
        sc, cam = scenes.tiny_workload()
    else:
        sc = scenes.cube_scene(300, seed=7, sh_degree=0, beta_range=(0.3, 16.0), beta_log=True)
        cam = scenes.tiny_camera(45, 37)
    k = oracle.keys(sc, cam)
    kk, vv = oracle.sorted_keys(sc, cam, key_info=k)
    tx = (cam.width + 15) // 16
    listed = {}
    for key, g in zip(kk, vv):
        listed.setdefault(int(g), set()).add(int(key >> np.uint64(32)))
    margin_abs, margin_rel = 1e-2, float(np.float32(1e-3))
    n_checked = 0
    for g in np.nonzero(k["touched"])[0]:
        a, b, c = (float(x) for x in k["cov2d"][g])
        det = a * c - b * b
        conic = (c / det, -b / det, a / det)
        u, v = (float(x) for x in k["mean2d"][g])
        qlim = float(k["qstar"][g]) * (1 + margin_rel) ** 2
        r = k["rect"][g]
        tiles = listed.get(int(g), set())
        assert len(tiles) == int(k["touched"][g])
        for ty in range(r[1], r[3]):
            for tx_ in range(r[0], r[2]):
                t = ty * tx + tx_
                x0, y0 = 16.0 * tx_, 16.0 * ty
                if t in tiles:   # the ellipse, widened by the margin in x, meets the tile
                    q = _qmin_over_box(conic, u, v, x0 - margin_abs - 1e-3, x0 + 16 + margin_abs + 1e-3, y0, y0 + 16)
                    assert q <= qlim * (1 + 1e-4), (g, t, q, qlim)
                else:            # it does not meet the tile
                    q = _qmin_over_box(conic, u, v, x0, x0 + 16, y0, y0 + 16)
                    assert q >= qlim * (1 - 1e-4), (g, t, q, qlim)
                n_checked += 1
    assert n_checked > 1000


# ---------------------------------------------------------------- gradients
def _fd_check(sc, cam, params, seed, n_check_prims=None, h=1e-6):
    rng = np.random.default_rng(seed)
    base = oracle.render(sc, cam, params=params)
    g = rng.standard_normal(base["img"].shape)
    g *= (base["flags"] == 0)[None]
    an = oracle.backward(sc, cam, g, params=params)
    names = ["means", "scales", "quats", "betas", "opacities", "shs"]
    prims = range(sc.n) if n_check_prims is None else rng.choice(sc.n, n_check_prims, replace=False)

    def loss(s2):
        return float((oracle.render(s2, cam, params=params)["img"] * g).sum())

    for name in names:
        fd = []
        ref = []
        for i in prims:
            arr = getattr(sc, name)
            width = arr.reshape(arr.shape[0], -1).shape[1]
            for j in range(width):
                vals = []
                for sgn in (+1, -1):
                    s2 = scenes.Scene(*(a.copy() for a in sc.arrays()), sc.sh_degree)
                    a2 = getattr(s2, name)
                    a2.reshape(a2.shape[0], -1)[i, j] += sgn * h
                    vals.append(loss(s2))
                fd.append((vals[0] - vals[1]) / (2 * h))
                ref.append(an[name].reshape(an[name].shape[0], -1)[i, j])
        fd, ref = np.array(fd), np.array(ref)
        assert rel_err(ref, fd) < 1e-6, (name, rel_err(ref, fd))


def _f64(sc):
    return scenes.Scene(*(np.asarray(a, np.float64) for a in sc.arrays()), sc.sh_degree)


@pytest.mark.parametrize("mode,phi_mode", [(oracle.MODE_GEF, 0), (oracle.MODE_PAPER_APPROX, 0),
                                           (oracle.MODE_GEF, 1), (oracle.MODE_GEF, 2)])
def test_backward_matches_finite_differences(mode, phi_mode):
    sc = _f64(random_small_scene(10, seed=21, beta_range=(0.6, 4.5) if phi_mode == 0 else (1.2, 4.5)))
    cam = axis_camera(32, 32, bg=(0.2, 0.1, 0.3))
    _fd_check(sc, cam, dict(mode=mode, phi_mode=phi_mode), seed=1)


def test_backward_matches_finite_differences_sh3_offaxis():
    sc = _f64(random_small_scene(6, seed=22, beta_range=(1.2, 3.0), degree=3))
    cam = scenes.look_at((0.4, 0.3, -0.5), (0.0, 0.0, 4.5), (0.0, -1.0, 0.0), 32, 28, 70.0)
    _fd_check(sc, cam, None, seed=2)


def _geometry_cases():
    off = scenes.cube_scene(2000, seed=17, beta_range=(0.5, 8.0), beta_log=True, scale_range=(0.02, 0.3))
    # camera aimed past the cube's edge: many primitives' centres and ellipses lie partly off the image
    off_cam = scenes.look_at((2.2, 0.8, -3.0), (2.2, 0.8, 0.0), (0.0, -1.0, 0.0), 96, 64, 60.0)
    return {
        "tiny": (*scenes.tiny_workload(), None),
        "wide_beta_ragged": (scenes.cube_scene(300, seed=11, beta_range=(0.3, 16.0), beta_log=True,
                                               scale_range=(0.02, 0.2)), scenes.tiny_camera(45, 37), None),
        "exact_phi": (scenes.cube_scene(400, seed=14, beta_range=(0.8, 12.0), beta_log=True,
                                        scale_range=(0.01, 0.06)), scenes.tiny_camera(70, 50), dict(phi_mode=1)),
        "paper_form": (*scenes.tiny_workload(), dict(mode=1)),
        "off_image": (off, off_cam, None),
    }


@pytest.mark.parametrize("which", list(_geometry_cases()))
def test_tile_lists_against_fp64_geometry(which):
    """The key module's lists against the extent ellipse in FP64 (oracle.project's conic, q* from
    libm), with none of the key path's FP32 arithmetic: complete (every tile the ellipse meets is
    listed) and tight (every listed tile meets the ellipse widened by the stated margins).  The
    off-image case pins that a row whose part of the ellipse lies wholly off the image lists no
    tile.  The depth keys against the FP64 camera depth, and each tile's order against it."""
    from helpers import check_depth_keys_fp64, check_tile_lists_fp64
    sc, cam, p = _geometry_cases()[which]
    k = oracle.keys(sc, cam, p)
    kk, vv = oracle.sorted_keys(sc, cam, p, key_info=k)
    n, fails = check_tile_lists_fp64(sc, cam, p, kk, vv, oracle)
    assert n > 1000 and not fails, fails
    assert not check_depth_keys_fp64(sc, cam, k["depth_key"], oracle, kk, vv)


def test_gradient_rounding_scale():
    """The oracle's per-element rounding scale (``cond``): for the 2D gradients the sum over pixels
    of the absolute per-pixel contributions, for the parameters those sums carried through the
    absolute Jacobian.  Pinned by: a single pixel, where it equals the absolute 2D gradient and
    bounds the parameter gradients; the triangle inequality (cond >= |g| everywhere); additivity
    over disjoint pixel sets; and an exact cancellation, two pixels symmetric about a lone
    isotropic splat's centre, whose x-mean gradients cancel while their magnitudes add."""
    sc, cam = scenes.tiny_workload()
    ref = oracle.render(sc, cam)
    rng = np.random.default_rng(3)
    ok = np.nonzero(ref["flags"].reshape(-1) == 0)[0]
    pix = rng.choice(ok, 40, replace=False)
    g = rng.standard_normal((3, pix.size))
    full = oracle.backward(sc, cam, g, pixels=pix, cond=True)
    for k in ("means", "scales", "quats", "betas", "opacities", "shs", "inter"):
        assert np.all(full["cond"][k] >= np.abs(full[k]) * (1 - 1e-12)), k
    a = oracle.backward(sc, cam, g[:, :17], pixels=pix[:17], cond=True)
    b = oracle.backward(sc, cam, g[:, 17:], pixels=pix[17:], cond=True)
    np.testing.assert_allclose(a["cond"]["inter"] + b["cond"]["inter"], full["cond"]["inter"], rtol=1e-12, atol=0)
    one = oracle.backward(sc, cam, g[:, :1], pixels=pix[:1], cond=True)
    np.testing.assert_allclose(one["cond"]["inter"], np.abs(one["inter"]), rtol=1e-15, atol=0)
    for k in ("means", "scales", "quats", "opacities"):
        assert np.all(one["cond"][k] >= np.abs(one[k]) * (1 - 1e-12))
    # exact cancellation: an isotropic splat on the axis of a 64x64 camera projects to (32, 32);
    # pixels (31, 32) and (32, 32) sit at dx = -0.5 and +0.5, dy = +0.5
    lone = make_scene([[0.0, 0.0, 4.0]], [0.2, 0.2, 0.2], [1.0, 0.0, 0.0, 0.0], [2.0], [0.8], rgb=[[0.6, 0.3, 0.2]])
    cam2 = axis_camera(64, 64)
    two = np.array([32 * 64 + 31, 32 * 64 + 32])
    r = oracle.backward(lone, cam2, np.ones((3, 2)), pixels=two, cond=True)
    s1 = oracle.backward(lone, cam2, np.ones((3, 1)), pixels=two[:1], cond=True)
    assert abs(r["inter"][0, 0]) <= 1e-12 * abs(s1["inter"][0, 0])
    np.testing.assert_allclose(r["cond"]["inter"][0, 0], 2 * abs(s1["inter"][0, 0]), rtol=1e-12)
